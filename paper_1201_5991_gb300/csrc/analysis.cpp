// Host-side index analysis of one BDDC level; see analysis.h.
//
// Readings of the paper taken here (Algorithm 1 names the steps but not their rules):
//   * interface node: contained in >= 2 subdomains;
//   * glob: maximal set of interface nodes with identical sharing sets, split into
//     components connected through shared (pseudo-)elements; globs ordered by smallest node;
//   * kind: 2 sharing subdomains -> face (3D) / edge (2D); >= 3 -> vertex if the glob is one
//     node, edge otherwise;
//   * corners = vertex globs, plus nodes promoted by a rigid-body sufficiency test (a scalar
//     problem needs one constrained point, 2D elasticity two distinct points, 3D elasticity
//     three non-collinear points; constrained points are centroids of globs constrained in
//     every component and nodes whose DOFs are all prescribed);
//   * one coarse DOF per constrained glob and component present on it; its constraint row
//     is the arithmetic average of that component over the glob's free DOFs (Sec. 2, Sec. 4).
#include "analysis.h"

#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <atomic>
#include <cmath>
#include <functional>
#include <numeric>
#include <thread>
#include <unordered_map>

namespace bddc {

namespace {

int64_t find_root(std::vector<int64_t>& parent, int64_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

bool same_set(const LevelMaps& m, int64_t a, int64_t b) {
  int64_t la = m.node_sub_ptr[a + 1] - m.node_sub_ptr[a];
  int64_t lb = m.node_sub_ptr[b + 1] - m.node_sub_ptr[b];
  if (la != lb) return false;
  return std::equal(m.node_sub.begin() + m.node_sub_ptr[a], m.node_sub.begin() + m.node_sub_ptr[a + 1],
                    m.node_sub.begin() + m.node_sub_ptr[b]);
}

struct Pt {
  double x[3];
};

double dist2(const Pt& a, const Pt& b, int dim) {
  double s = 0.0;
  for (int d = 0; d < dim; ++d) {
    double t = a.x[d] - b.x[d];
    s = s + t * t;
  }
  return s;
}

// |(p - o) x u| for 3D points
double cross_norm(const Pt& p, const Pt& o, const double* u) {
  double a0 = p.x[0] - o.x[0], a1 = p.x[1] - o.x[1], a2 = p.x[2] - o.x[2];
  double c0 = a1 * u[2] - a2 * u[1];
  double c1 = a2 * u[0] - a0 * u[2];
  double c2 = a0 * u[1] - a1 * u[0];
  return std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

constexpr unsigned kWorkers = kHostWorkers;

void parallel_range_worker(int64_t n, const std::function<void(int64_t, int)>& fn) { host_parallel(n, fn); }

void parallel_range(int64_t n, const std::function<void(int64_t)>& fn) {
  parallel_range_worker(n, [&](int64_t i, int) { fn(i); });
}

}  // namespace

bool analyze_level(const LevelMesh& mesh, unsigned constraints, bool all_corners, LevelMaps* out,
                   std::string* err) {
  LevelMaps& m = *out;
  m = LevelMaps();
  const int64_t nn = mesh.n_nodes, ne = mesh.n_elems, ns = mesh.n_sub;
  const int dim = mesh.dim, nc = mesh.ncomp;
  if (ns <= 0 || ne <= 0) {
    *err = "empty mesh or partition";
    return false;
  }
  // subdomain -> elements (ascending)
  m.sub_elem_ptr.assign(ns + 1, 0);
  for (int64_t e = 0; e < ne; ++e) {
    int32_t s = mesh.part[e];
    if (s < 0 || s >= ns) {
      *err = "partition id out of range at element " + std::to_string(e);
      return false;
    }
    m.sub_elem_ptr[s + 1]++;
  }
  for (int64_t s = 0; s < ns; ++s) {
    if (m.sub_elem_ptr[s + 1] == 0) {
      *err = "empty subdomain " + std::to_string(s);
      return false;
    }
    m.sub_elem_ptr[s + 1] += m.sub_elem_ptr[s];
  }
  m.sub_elems.resize(ne);
  {
    std::vector<int64_t> fill(m.sub_elem_ptr.begin(), m.sub_elem_ptr.end() - 1);
    for (int64_t e = 0; e < ne; ++e) m.sub_elems[fill[mesh.part[e]]++] = e;
  }
  // subdomain -> nodes (sorted unique)
  {   // connectivity check in chunks on the host pool; the first bad entry is reported
    constexpr int64_t kChunk = 65536;
    const int64_t nq = (int64_t)mesh.en.size();
    std::atomic<int64_t> bad{INT64_MAX};
    parallel_range((nq + kChunk - 1) / kChunk, [&](int64_t b) {
      for (int64_t q = b * kChunk; q < std::min(nq, (b + 1) * kChunk); ++q)
        if (mesh.en[q] < 0 || mesh.en[q] >= nn) {
          int64_t cur = bad.load();
          while (q < cur && !bad.compare_exchange_weak(cur, q)) {
          }
          break;
        }
    });
    if (bad.load() != INT64_MAX) {
      *err = "node id out of range in element connectivity entry " + std::to_string(bad.load());
      return false;
    }
  }
  std::vector<std::vector<int64_t>> sub_nodes(ns);
  std::vector<std::vector<char>> seen(kWorkers);   // per worker: node already listed
  parallel_range_worker(ns, [&](int64_t s, int w) {
    auto& v = sub_nodes[s];
    std::vector<char>& mk = seen[w];
    if ((int64_t)mk.size() < nn) mk.assign(nn, 0);
    for (int64_t k = m.sub_elem_ptr[s]; k < m.sub_elem_ptr[s + 1]; ++k) {
      int64_t e = m.sub_elems[k];
      for (int64_t q = mesh.en_ptr[e]; q < mesh.en_ptr[e + 1]; ++q) {
        const int64_t p = mesh.en[q];
        if (!mk[p]) {
          mk[p] = 1;
          v.push_back(p);
        }
      }
    }
    for (int64_t p : v) mk[p] = 0;
    std::sort(v.begin(), v.end());
  });
  // node -> sharing set (ascending subdomain ids)
  m.node_sub_ptr.assign(nn + 1, 0);
  for (int64_t s = 0; s < ns; ++s)
    for (int64_t p : sub_nodes[s]) m.node_sub_ptr[p + 1]++;
  for (int64_t p = 0; p < nn; ++p) m.node_sub_ptr[p + 1] += m.node_sub_ptr[p];
  m.node_sub.resize(m.node_sub_ptr[nn]);
  {
    std::vector<int64_t> fill(m.node_sub_ptr.begin(), m.node_sub_ptr.end() - 1);
    for (int64_t s = 0; s < ns; ++s)
      for (int64_t p : sub_nodes[s]) m.node_sub[fill[p]++] = (int32_t)s;
  }
  auto nsh = [&](int64_t p) { return m.node_sub_ptr[p + 1] - m.node_sub_ptr[p]; };
  std::vector<char> iface(nn, 0);
  for (int64_t p = 0; p < nn; ++p) iface[p] = nsh(p) >= 2;

  // globs: union of interface nodes with equal sharing sets inside an element
  std::vector<int64_t> parent(nn);
  std::iota(parent.begin(), parent.end(), 0);
  if (!all_corners) {
    // the pairs to join are found per chunk of elements in parallel and joined afterwards: a
    // component's root is always its smallest node, so the globs do not depend on the order
    const int64_t chunk = 4096, nchunk = (ne + chunk - 1) / chunk;
    std::vector<std::vector<std::pair<int64_t, int64_t>>> joins(nchunk);
    parallel_range(nchunk, [&](int64_t b) {
      std::vector<int64_t> firsts;
      for (int64_t e = b * chunk; e < std::min(ne, (b + 1) * chunk); ++e) {
        firsts.clear();
        for (int64_t q = mesh.en_ptr[e]; q < mesh.en_ptr[e + 1]; ++q) {
          int64_t p = mesh.en[q];
          if (!iface[p]) continue;
          int64_t rep = -1;
          for (int64_t f : firsts)
            if (same_set(m, f, p)) {
              rep = f;
              break;
            }
          if (rep < 0)
            firsts.push_back(p);
          else
            joins[b].emplace_back(p, rep);
        }
      }
    });
    for (const auto& jb : joins)
      for (const auto& pr : jb) {
        int64_t a = find_root(parent, pr.first), b = find_root(parent, pr.second);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
      }
  }
  // number globs by first (= smallest) node
  std::vector<int64_t> glob_of_root(nn, -1);
  std::vector<int64_t> node_glob(nn, -1);
  int64_t n_globs = 0;
  for (int64_t p = 0; p < nn; ++p) {
    if (!iface[p]) continue;
    int64_t r = find_root(parent, p);
    if (glob_of_root[r] < 0) glob_of_root[r] = n_globs++;
    node_glob[p] = glob_of_root[r];
  }
  m.glob_ptr.assign(n_globs + 1, 0);
  for (int64_t p = 0; p < nn; ++p)
    if (node_glob[p] >= 0) m.glob_ptr[node_glob[p] + 1]++;
  for (int64_t g = 0; g < n_globs; ++g) m.glob_ptr[g + 1] += m.glob_ptr[g];
  m.glob_nodes.resize(m.glob_ptr[n_globs]);
  {
    std::vector<int64_t> fill(m.glob_ptr.begin(), m.glob_ptr.end() - 1);
    for (int64_t p = 0; p < nn; ++p)
      if (node_glob[p] >= 0) m.glob_nodes[fill[node_glob[p]]++] = p;
  }
  m.glob_kind.resize(n_globs);
  m.glob_promoted.assign(n_globs, 0);
  for (int64_t g = 0; g < n_globs; ++g) {
    int64_t p0 = m.glob_nodes[m.glob_ptr[g]];
    int64_t cnt = m.glob_ptr[g + 1] - m.glob_ptr[g];
    if (all_corners)
      m.glob_kind[g] = kVertex;
    else if (nsh(p0) == 2)
      m.glob_kind[g] = dim == 3 ? kFace : kEdge;
    else
      m.glob_kind[g] = cnt == 1 ? kVertex : kEdge;
  }

  auto node_has_free = [&](int64_t p) {
    for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q)
      if (mesh.nd_id[q] >= 0) return true;
    return false;
  };
  const uint32_t rmask = mesh.rigid_mask;
  // a node's rigid-mode DOFs: all prescribed (a constrained point) / all present and free
  auto node_all_prescribed = [&](int64_t p) {
    bool any = false;
    for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q) {
      if (!((rmask >> mesh.nd_comp[q]) & 1u)) continue;
      any = true;
      if (mesh.nd_id[q] >= 0) return false;
    }
    return any;
  };
  auto node_all_free_full = [&](int64_t p) {
    uint32_t present = 0;
    for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q) {
      if (!((rmask >> mesh.nd_comp[q]) & 1u)) continue;
      if (mesh.nd_id[q] < 0) return false;
      present |= 1u << mesh.nd_comp[q];
    }
    return present == rmask;
  };
  auto constrained = [&](int64_t g) -> bool {
    if (m.glob_promoted[g]) return true;
    unsigned bit = m.glob_kind[g] == kVertex ? 1u : (m.glob_kind[g] == kEdge ? 2u : 4u);
    return (constraints & bit) != 0;
  };
  // per glob: components with a free DOF (bitmask), centroid of the nodes carrying free DOFs
  std::vector<uint32_t> glob_comps;
  auto add_glob_info = [&](int64_t g) {
    uint32_t mask = 0;
    for (int64_t k = m.glob_ptr[g]; k < m.glob_ptr[g + 1]; ++k) {
      int64_t p = m.glob_nodes[k];
      for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q)
        if (mesh.nd_id[q] >= 0) mask |= 1u << mesh.nd_comp[q];
    }
    glob_comps.push_back(mask);
    double c[3] = {0, 0, 0};
    int64_t cnt = 0;
    for (int pass = 0; pass < 2 && cnt == 0; ++pass) {
      for (int64_t k = m.glob_ptr[g]; k < m.glob_ptr[g + 1]; ++k) {
        int64_t p = m.glob_nodes[k];
        if (pass == 0 && !node_has_free(p)) continue;
        for (int d = 0; d < dim; ++d) c[d] = c[d] + mesh.coords[p * dim + d];
        ++cnt;
      }
    }
    for (int d = 0; d < dim; ++d) m.glob_centroid.push_back(c[d] / (double)cnt);
  };
  for (int64_t g = 0; g < n_globs; ++g) add_glob_info(g);

  // subdomain -> globs touching it (ascending glob index); promoted globs appended later
  std::vector<std::vector<int64_t>> sub_globs(ns);
  for (int64_t g = 0; g < n_globs; ++g) {
    int64_t p0 = m.glob_nodes[m.glob_ptr[g]];
    for (int64_t k = m.node_sub_ptr[p0]; k < m.node_sub_ptr[p0 + 1]; ++k) sub_globs[m.node_sub[k]].push_back(g);
  }

  // corner selection with the rigid-body sufficiency test
  std::vector<char> is_corner(nn, 0);
  for (int64_t g = 0; g < n_globs; ++g)
    if (m.glob_kind[g] == kVertex && constrained(g)) is_corner[m.glob_nodes[m.glob_ptr[g]]] = 1;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t p = 0; p < nn; ++p)
    for (int d = 0; d < dim; ++d) {
      lo[d] = std::min(lo[d], mesh.coords[p * dim + d]);
      hi[d] = std::max(hi[d], mesh.coords[p * dim + d]);
    }
  double diam2 = 0.0;
  for (int d = 0; d < dim; ++d) diam2 = diam2 + (hi[d] - lo[d]) * (hi[d] - lo[d]);
  const double tol = 1e-12 * diam2;

  std::vector<Pt> pts;
  auto gather_points_into = [&](int64_t s, std::vector<Pt>& out) {
    out.clear();
    for (int64_t g : sub_globs[s]) {
      if (!constrained(g) || (glob_comps[g] & rmask) != rmask) continue;
      Pt q{{0, 0, 0}};
      for (int d = 0; d < dim; ++d) q.x[d] = m.glob_centroid[g * dim + d];
      out.push_back(q);
    }
    for (int64_t p : sub_nodes[s]) {
      if (!node_all_prescribed(p)) continue;
      Pt q{{0, 0, 0}};
      for (int d = 0; d < dim; ++d) q.x[d] = mesh.coords[p * dim + d];
      out.push_back(q);
    }
  };
  auto gather_points = [&](int64_t s) { gather_points_into(s, pts); };
  auto sufficient_for = [&](const std::vector<Pt>& q) -> bool {
    if (mesh.rigid_points == 1) return !q.empty();
    if (q.empty()) return false;
    size_t j = 0;
    double best = -1.0;
    for (size_t k = 0; k < q.size(); ++k) {
      double d = std::sqrt(dist2(q[k], q[0], dim));
      if (d > best) {
        best = d;
        j = k;
      }
    }
    if (mesh.rigid_points == 2) return best * best > tol;
    if (best * best <= tol) return false;
    double u[3] = {q[j].x[0] - q[0].x[0], q[j].x[1] - q[0].x[1], q[j].x[2] - q[0].x[2]};
    double mx = 0.0;
    for (size_t k = 0; k < q.size(); ++k) mx = std::max(mx, cross_norm(q[k], q[0], u));
    return mx > tol;
  };
  auto sufficient = [&]() -> bool { return sufficient_for(pts); };
  // the test of every subdomain on the initial constraints, in parallel (0: insufficient,
  // 1: sufficient, 2: no interface node); the ordered pass below reuses it until the first
  // promotion changes the constraints of later subdomains
  std::vector<char> pre(ns, 0);
  parallel_range(ns, [&](int64_t s) {
    bool has_iface = false;
    for (int64_t p : sub_nodes[s]) has_iface = has_iface || iface[p];
    if (!has_iface) {
      pre[s] = 2;
      return;
    }
    std::vector<Pt> local;
    gather_points_into(s, local);
    pre[s] = sufficient_for(local) ? 1 : 0;
  });
  bool promoted_any = false;
  for (int64_t s = 0; s < ns; ++s) {
    if (pre[s] == 2) continue;   // the whole (connected) problem: nothing to constrain
    if (!promoted_any && pre[s] == 1) continue;
    int tries = 0;
    for (;;) {
      gather_points(s);
      if (sufficient()) break;
      if (++tries > 16) {
        *err = "corner selection did not terminate on subdomain " + std::to_string(s);
        return false;
      }
      std::vector<int64_t> cand;
      for (int64_t p : sub_nodes[s])
        if (iface[p] && !is_corner[p] && node_all_free_full(p)) cand.push_back(p);
      if (cand.empty()) {
        *err = "no candidate corner in subdomain " + std::to_string(s);
        return false;
      }
      int64_t pick = cand[0];
      if (!pts.empty()) {
        size_t j = 0;
        double best = -1.0;
        for (size_t k = 0; k < pts.size(); ++k) {
          double d = std::sqrt(dist2(pts[k], pts[0], dim));
          if (d > best) {
            best = d;
            j = k;
          }
        }
        double u[3] = {0, 0, 0};
        bool use_line = !(best * best <= tol || mesh.rigid_points <= 2);
        if (use_line)
          for (int d = 0; d < 3; ++d) u[d] = (pts[j].x[d] - pts[0].x[d]) / best;
        double bd = -1.0;
        for (int64_t p : cand) {
          Pt q{{0, 0, 0}};
          for (int d = 0; d < dim; ++d) q.x[d] = mesh.coords[p * dim + d];
          double d = use_line ? cross_norm(q, pts[0], u) : std::sqrt(dist2(q, pts[0], dim));
          if (d > bd) {
            bd = d;
            pick = p;
          }
        }
      }
      // append a promoted corner glob {pick}
      int64_t g = (int64_t)m.glob_kind.size();
      m.glob_nodes.push_back(pick);
      m.glob_ptr.push_back((int64_t)m.glob_nodes.size());
      m.glob_kind.push_back(kVertex);
      m.glob_promoted.push_back(1);
      add_glob_info(g);
      for (int64_t k = m.node_sub_ptr[pick]; k < m.node_sub_ptr[pick + 1]; ++k) sub_globs[m.node_sub[k]].push_back(g);
      is_corner[pick] = 1;
      m.n_promoted++;
      promoted_any = true;
    }
  }
  n_globs = (int64_t)m.glob_kind.size();

  // coarse DOFs in (glob order, component)
  m.glob_coarse_ptr.assign(n_globs + 1, 0);
  for (int64_t g = 0; g < n_globs; ++g) {
    if (constrained(g))
      for (int c = 0; c < nc; ++c)
        if (glob_comps[g] & (1u << c)) {
          m.coarse_glob.push_back(g);
          m.coarse_comp.push_back(c);
        }
    m.glob_coarse_ptr[g + 1] = (int64_t)m.coarse_glob.size();
  }
  m.n_coarse = (int64_t)m.coarse_glob.size();

  // global interface numbering: the interface nodes' DOFs in node order (counted and written by
  // node chunks on the host pool, offsets scanned in chunk order), then sorted by id
  constexpr int64_t kNodeChunk = 4096;
  const int64_t nchunk = (nn + kNodeChunk - 1) / kNodeChunk;
  {
    std::vector<int64_t> cnt(nchunk + 1, 0);
    parallel_range(nchunk, [&](int64_t b) {
      int64_t c = 0;
      for (int64_t p = b * kNodeChunk; p < std::min(nn, (b + 1) * kNodeChunk); ++p)
        if (iface[p])
          for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q) c += mesh.nd_id[q] >= 0;
      cnt[b + 1] = c;
    });
    for (int64_t b = 0; b < nchunk; ++b) cnt[b + 1] += cnt[b];
    m.iface_dofs.resize(cnt[nchunk]);
    parallel_range(nchunk, [&](int64_t b) {
      int64_t w = cnt[b];
      for (int64_t p = b * kNodeChunk; p < std::min(nn, (b + 1) * kNodeChunk); ++p)
        if (iface[p])
          for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q)
            if (mesh.nd_id[q] >= 0) m.iface_dofs[w++] = mesh.nd_id[q];
    });
  }
  if (!std::is_sorted(m.iface_dofs.begin(), m.iface_dofs.end()))   // level 1 numbers DOFs node by node
    std::sort(m.iface_dofs.begin(), m.iface_dofs.end());
  m.n_iface = (int64_t)m.iface_dofs.size();
  std::vector<int64_t> iface_pos(mesh.n_dof, -1);
  parallel_range((m.n_iface + kNodeChunk - 1) / kNodeChunk, [&](int64_t b) {
    for (int64_t k = b * kNodeChunk; k < std::min(m.n_iface, (b + 1) * kNodeChunk); ++k) iface_pos[m.iface_dofs[k]] = k;
  });

  // per-subdomain local orderings, weights, constraint rows (computed per subdomain in
  // parallel, then concatenated in subdomain order)
  std::vector<int64_t> dof_node(mesh.n_dof, -1);
  parallel_range(nchunk, [&](int64_t b) {   // every DOF id belongs to one node: disjoint writes
    for (int64_t p = b * kNodeChunk; p < std::min(nn, (b + 1) * kNodeChunk); ++p)
      for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q)
        if (mesh.nd_id[q] >= 0) dof_node[mesh.nd_id[q]] = p;
  });
  struct SubOut {
    std::vector<int64_t> interior, inter, coarse, crow_len, ccol;
  };
  std::vector<SubOut> so(ns);
  // sort key: DOFs of the last component (Stokes pressures) after the others, then id
  const int64_t shift = (int64_t)1 << 40;
  auto key_of = [&](int64_t q) { return mesh.nd_id[q] + (mesh.nd_comp[q] == mesh.last_comp ? shift : 0); };
  parallel_range(ns, [&](int64_t s) {
    SubOut& o = so[s];
    for (int64_t p : sub_nodes[s])
      for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q) {
        if (mesh.nd_id[q] < 0) continue;
        (iface[p] ? o.inter : o.interior).push_back(key_of(q));
      }
    // nodes come in ascending order and DOF ids grow with (node, component), so the keys are
    // usually ordered already (not when the last component is moved to the end)
    if (!std::is_sorted(o.interior.begin(), o.interior.end())) std::sort(o.interior.begin(), o.interior.end());
    if (!std::is_sorted(o.inter.begin(), o.inter.end())) std::sort(o.inter.begin(), o.inter.end());
    const int64_t nI = (int64_t)o.interior.size();
    // constraint rows: globs touching s in glob order -> ascending coarse ids; their DOFs are
    // interface DOFs, found in the sorted interface keys
    std::vector<int64_t> gl = sub_globs[s];
    std::sort(gl.begin(), gl.end());
    for (int64_t g : gl)
      for (int64_t k = m.glob_coarse_ptr[g]; k < m.glob_coarse_ptr[g + 1]; ++k) {
        const int c = m.coarse_comp[k];
        o.coarse.push_back(k);
        const int64_t first = (int64_t)o.ccol.size();
        for (int64_t t = m.glob_ptr[g]; t < m.glob_ptr[g + 1]; ++t) {
          const int64_t p = m.glob_nodes[t];
          for (int64_t q = mesh.nd_ptr[p]; q < mesh.nd_ptr[p + 1]; ++q)
            if (mesh.nd_comp[q] == c && mesh.nd_id[q] >= 0) {
              const int64_t key = key_of(q);
              const int64_t pos = std::lower_bound(o.inter.begin(), o.inter.end(), key) - o.inter.begin();
              o.ccol.push_back(nI + pos);
            }
        }
        o.crow_len.push_back((int64_t)o.ccol.size() - first);
      }
    for (auto& k : o.interior) k %= shift;
    for (auto& k : o.inter) k %= shift;
  });
  // offsets, then every subdomain's block filled in parallel
  m.sub_dof_ptr.assign(ns + 1, 0);
  m.sub_coarse_ptr.assign(ns + 1, 0);
  std::vector<int64_t> ccol_off(ns + 1, 0);
  m.sub_nI.resize(ns);
  for (int64_t s = 0; s < ns; ++s) {
    m.sub_dof_ptr[s + 1] = m.sub_dof_ptr[s] + (int64_t)(so[s].interior.size() + so[s].inter.size());
    m.sub_coarse_ptr[s + 1] = m.sub_coarse_ptr[s] + (int64_t)so[s].coarse.size();
    ccol_off[s + 1] = ccol_off[s] + (int64_t)so[s].ccol.size();
    m.sub_nI[s] = (int64_t)so[s].interior.size();
  }
  m.sub_dofs.resize(m.sub_dof_ptr[ns]);
  m.sub_iface.resize(m.sub_dof_ptr[ns]);
  m.sub_wmult.resize(m.sub_dof_ptr[ns]);
  m.sub_coarse.resize(m.sub_coarse_ptr[ns]);
  m.c_ptr.resize(m.sub_coarse_ptr[ns] + 1);
  m.c_col.resize(ccol_off[ns]);
  m.c_val.resize(ccol_off[ns]);
  m.c_ptr[0] = 0;
  parallel_range(ns, [&](int64_t s) {
    const SubOut& o = so[s];
    int64_t w = m.sub_dof_ptr[s];
    for (int64_t d : o.interior) {
      m.sub_dofs[w] = d;
      m.sub_iface[w] = -1;
      m.sub_wmult[w++] = 0.0;
    }
    for (int64_t d : o.inter) {
      m.sub_dofs[w] = d;
      m.sub_iface[w] = iface_pos[d];
      m.sub_wmult[w++] = 1.0 / (double)nsh(dof_node[d]);
    }
    int64_t t = ccol_off[s];
    for (size_t r = 0; r < o.coarse.size(); ++r) {
      const int64_t row = m.sub_coarse_ptr[s] + (int64_t)r;
      m.sub_coarse[row] = o.coarse[r];
      const int64_t cnt = o.crow_len[r];
      for (int64_t u = 0; u < cnt; ++u, ++t) {
        m.c_col[t] = o.ccol[t - ccol_off[s]];
        m.c_val[t] = 1.0 / (double)cnt;
      }
      m.c_ptr[row + 1] = t;
    }
  });
  return true;
}

void next_level_mesh(const LevelMesh& mesh, const LevelMaps& maps, const int32_t* part, int64_t n_sub_next,
                     LevelMesh* out) {
  LevelMesh& n = *out;
  n = LevelMesh();
  n.dim = mesh.dim;
  n.ncomp = mesh.ncomp;
  const int dim = mesh.dim;
  const int64_t G = maps.n_globs();
  std::vector<int64_t> node_of_glob(G, -1);
  n.nd_ptr.assign(1, 0);
  for (int64_t g = 0; g < G; ++g) {
    if (maps.glob_coarse_ptr[g + 1] == maps.glob_coarse_ptr[g]) continue;
    node_of_glob[g] = n.n_nodes++;
    for (int d = 0; d < dim; ++d) n.coords.push_back(maps.glob_centroid[g * dim + d]);
    for (int64_t k = maps.glob_coarse_ptr[g]; k < maps.glob_coarse_ptr[g + 1]; ++k) {
      n.nd_comp.push_back(maps.coarse_comp[k]);
      n.nd_id.push_back(k);
    }
    n.nd_ptr.push_back((int64_t)n.nd_id.size());
  }
  const int64_t ns = maps.n_sub();
  n.n_elems = ns;
  n.en_ptr.assign(1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t last = -1;
    for (int64_t k = maps.sub_coarse_ptr[s]; k < maps.sub_coarse_ptr[s + 1]; ++k) {
      int64_t cd = maps.sub_coarse[k];
      int64_t g = maps.coarse_glob[cd];
      if (g != last) {   // the subdomain's coarse DOFs come glob by glob, all components
        n.en.push_back(node_of_glob[g]);
        last = g;
      }
    }
    n.en_ptr.push_back((int64_t)n.en.size());
  }
  n.part.assign(part, part + ns);
  n.n_sub = n_sub_next;
  n.n_dof = maps.n_coarse;
  n.rigid_mask = mesh.rigid_mask;
  n.rigid_points = mesh.rigid_points;
  n.last_comp = mesh.last_comp;
}

// ------------------------------------------------------------------ host thread pool
namespace {

// Persistent workers (created on first use, kept for the life of the process): a parallel region
// publishes the job and an epoch under the mutex, the workers and the caller take iterations from
// one atomic counter, and the caller waits until every worker has left the region.  Spawning
// fresh threads for every region cost more than the short regions of a set-up themselves.
class HostPool {
 public:
  explicit HostPool(int nw) {
    for (int t = 1; t <= nw; ++t) th_.emplace_back([this, t]() { work(t); });
  }
  int workers() const { return (int)th_.size(); }
  void run(int64_t n, const std::function<void(int64_t, int)>& fn) {
    std::lock_guard<std::mutex> one(run_mu_);   // one region at a time (handles set up concurrently)
    {
      std::lock_guard<std::mutex> g(mu_);
      fn_ = &fn;
      n_ = n;
      next_.store(0);
      busy_ = (int)th_.size();
      ++epoch_;
    }
    cv_.notify_all();
    in_region() = true;
    for (int64_t i; (i = next_.fetch_add(1)) < n;) fn(i, 0);
    in_region() = false;
    std::unique_lock<std::mutex> g(mu_);
    done_.wait(g, [this]() { return busy_ == 0; });
    fn_ = nullptr;
  }
  static bool& in_region() {
    thread_local bool r = false;
    return r;
  }

 private:
  void work(int id) {
    uint64_t seen = 0;
    in_region() = true;   // a nested call from a worker runs serially
    for (;;) {
      const std::function<void(int64_t, int)>* fn;
      int64_t n;
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&]() { return epoch_ != seen; });
        seen = epoch_;
        fn = fn_;
        n = n_;
      }
      for (int64_t i; (i = next_.fetch_add(1)) < n;) (*fn)(i, id);
      std::lock_guard<std::mutex> g(mu_);
      if (--busy_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_, run_mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int64_t, int)>* fn_ = nullptr;
  int64_t n_ = 0;
  std::atomic<int64_t> next_{0};
  int busy_ = 0;
  uint64_t epoch_ = 0;
};

}  // namespace

void host_parallel(int64_t n, const std::function<void(int64_t, int)>& fn) {
  static HostPool* pool = []() {
    const unsigned hc = std::thread::hardware_concurrency();
    const int nt = (int)std::max(1u, std::min((unsigned)kHostWorkers, hc == 0 ? 1u : hc));
    return new HostPool(nt - 1);   // never destroyed: the workers sleep until the process exits
  }();
  if (n < 4 || pool->workers() == 0 || HostPool::in_region()) {
    for (int64_t i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  pool->run(n, fn);
}

}  // namespace bddc
