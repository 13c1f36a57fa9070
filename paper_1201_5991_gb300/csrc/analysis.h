// Host-side index analysis of one BDDC level (Algorithm 1 of the paper, without the
// numerical steps): sharing sets, interface classification into faces / edges / vertices,
// corner selection with a rigid-body sufficiency test, constraint rows C_i (corner values
// and arithmetic averages), coarse numbering R_Ci, local DOF orderings, multiplicity
// weights, and the pseudo-mesh of the next level whose "elements" are the subdomains and
// whose "nodes" are the globs carrying coarse DOFs.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace bddc {

// Host worker threads of the set-up, shared by the analysis and the preparation of the levels.
constexpr int kHostWorkers = 16;
// fn(i, w) for i in [0, n) (independent iterations) on the calling thread and up to
// kHostWorkers - 1 persistent pool threads; w < kHostWorkers names the thread, so that per-thread
// scratch can be indexed by it.  Small ranges, and calls from inside a parallel region, run on
// the calling thread alone.
void host_parallel(int64_t n, const std::function<void(int64_t, int)>& fn);

enum GlobKind { kVertex = 0, kEdge = 1, kFace = 2 };

// A (pseudo-)mesh.  Level 1: FE nodes and elements.  Level l > 1: globs of level l-1 as
// nodes and subdomains of level l-1 as elements.
struct LevelMesh {
  int dim = 3;
  int ncomp = 1;
  int64_t n_nodes = 0, n_elems = 0, n_sub = 0, n_dof = 0;
  std::vector<double> coords;          // [n_nodes * dim]
  std::vector<int64_t> nd_ptr;         // node -> its DOFs (CSR)
  std::vector<int32_t> nd_comp;        //   component of each node DOF
  std::vector<int64_t> nd_id;          //   level DOF id, -1 = prescribed
  std::vector<int64_t> en_ptr, en;     // element -> nodes; the element matrix's DOFs are the
                                       // DOFs of its nodes in this order (nd_id, -1 = prescribed)
  std::vector<int32_t> part;           // element -> subdomain
  uint32_t rigid_mask = 1u;            // components that carry the floating (rigid) modes
  int rigid_points = 1;                // constrained points needed: 1, 2 (2D elasticity), 3 (3D elasticity)
  int last_comp = -1;                  // component ordered after the others in local orders (-1: none)
};

struct LevelMaps {
  int64_t n_iface = 0, n_coarse = 0, n_promoted = 0;
  std::vector<int64_t> node_sub_ptr;   // node -> sharing set (ascending)
  std::vector<int32_t> node_sub;
  std::vector<int64_t> glob_ptr, glob_nodes;
  std::vector<int32_t> glob_kind, glob_promoted;
  std::vector<int64_t> glob_coarse_ptr;   // coarse DOFs of glob g: [ptr[g], ptr[g+1])
  std::vector<double> glob_centroid;      // [n_globs * dim]
  std::vector<int64_t> coarse_glob;
  std::vector<int32_t> coarse_comp;
  std::vector<int64_t> iface_dofs;        // ascending level DOF ids
  std::vector<int64_t> sub_elem_ptr, sub_elems;
  std::vector<int64_t> sub_dof_ptr, sub_dofs, sub_nI, sub_iface;
  std::vector<double> sub_wmult;
  std::vector<int64_t> sub_coarse_ptr, sub_coarse;
  std::vector<int64_t> c_ptr, c_col;
  std::vector<double> c_val;
  int64_t n_globs() const { return (int64_t)glob_kind.size(); }
  int64_t n_sub() const { return (int64_t)sub_nI.size(); }
};

// Analyse one level.  Returns false and fills *err on an invalid mesh/partition.
bool analyze_level(const LevelMesh& mesh, unsigned constraints, bool all_corners, LevelMaps* out,
                   std::string* err);

// Pseudo-mesh of level l+1 from level l (part: level-l subdomain -> level-(l+1) subdomain).
void next_level_mesh(const LevelMesh& mesh, const LevelMaps& maps, const int32_t* part,
                     int64_t n_sub_next, LevelMesh* out);

}  // namespace bddc
