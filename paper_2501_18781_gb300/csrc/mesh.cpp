// Meshes and DoF maps (host side, built once per mesh; Appendix B: continuous Lagrange
// elements on adaptively refined hexahedral meshes).
//
// Lattice: nodes sit on the lattice of spacing h_finest / k; a node's key is
// z (R+1)^2 + y (R+1) + x with R = k * (cells per axis on the finest level), so sorting by
// key is the lexicographic (z, y, x) DoF order.  A lattice node that lies on the closure of
// a leaf K without being one of K's nodes hangs: its value is K's Q_k interpolant there.
// With 2:1 balance such nodes sit at half of K's node spacing, so the weights are products
// of 1D Lagrange values at p / 2k, p = 0..2k (dyadic rationals, exact in binary64).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <unordered_map>

#include "internal.h"

namespace mf {

namespace {

inline int64_t key_of(int64_t x, int64_t y, int64_t z, int64_t R) { return (z * (R + 1) + y) * (R + 1) + x; }

inline uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

// l_a(p / (2k)) for the degree-k equispaced Lagrange basis, by the product formula.
double lagrange_at_half_step(int k, int a, int p) {
  double x = double(p) / double(2 * k);
  double v = 1.0;
  for (int b = 0; b <= k; ++b) {
    if (b == a) continue;
    double xa = double(a) / double(k), xb = double(b) / double(k);
    v *= (x - xb) / (xa - xb);
  }
  return v;
}

void build_dirichlet_lists(mf_dofmap* m) {
  m->dirichlet.assign(m->n_dofs, 0);
  m->dirichlet_list.clear();
  if (!m->dirichlet_faces) return;
  const int64_t R = m->R[0];
  for (int64_t d = 0; d < m->n_dofs; ++d) {
    int64_t key = m->free_keys.empty() ? d : m->free_keys[d];
    int64_t x = key % (R + 1), y = (key / (R + 1)) % (R + 1), z = key / ((R + 1) * (R + 1));
    int64_t c[3] = {x, y, z};
    bool on = false;
    for (int ax = 0; ax < 3; ++ax) {
      if ((m->dirichlet_faces >> (2 * ax)) & 1u) on |= (c[ax] == 0);
      if ((m->dirichlet_faces >> (2 * ax + 1)) & 1u) on |= (c[ax] == m->R[ax]);
    }
    if (on) {
      m->dirichlet[d] = 1;
      m->dirichlet_list.push_back(int32_t(d));
    }
  }
}

}  // namespace

mf_status build_uniform_dofmap(mf_dofmap* m) {
  const mf_mesh* me = m->mesh;
  int k = m->degree;
  m->uniform = true;
  m->n_cells = int64_t(me->n[0]) * me->n[1] * me->n[2];
  for (int d = 0; d < 3; ++d) m->R[d] = int64_t(k) * me->n[d];
  m->n_dofs = (m->R[0] + 1) * (m->R[1] + 1) * (m->R[2] + 1);
  if (m->n_dofs >= (int64_t(1) << 31)) return fail(MF_EINVAL, "uniform map exceeds 2^31 DoFs");
  m->free_keys.clear();
  // Dirichlet DoFs: only the box faces; walk them instead of all nodes.
  m->dirichlet.assign(m->n_dofs, 0);
  m->dirichlet_list.clear();
  const int64_t Rx = m->R[0] + 1, Ry = m->R[1] + 1;
  if (m->dirichlet_faces) {
    for (int64_t z = 0; z <= m->R[2]; ++z)
      for (int64_t y = 0; y <= m->R[1]; ++y)
        for (int64_t x = 0; x <= m->R[0]; ++x) {
          bool interior = x > 0 && x < m->R[0] && y > 0 && y < m->R[1] && z > 0 && z < m->R[2];
          if (interior) { x = m->R[0] - 1; continue; }
          int64_t c[3] = {x, y, z};
          bool on = false;
          for (int ax = 0; ax < 3; ++ax) {
            if ((m->dirichlet_faces >> (2 * ax)) & 1u) on |= (c[ax] == 0);
            if ((m->dirichlet_faces >> (2 * ax + 1)) & 1u) on |= (c[ax] == m->R[ax]);
          }
          if (on) {
            int64_t d = x + Rx * (y + Ry * z);
            m->dirichlet[d] = 1;
            m->dirichlet_list.push_back(int32_t(d));
          }
        }
  }
  return MF_OK;
}

mf_status build_octree_dofmap(mf_dofmap* m) {
  const mf_mesh* me = m->mesh;
  const int k = m->degree, L = me->levels, nb = m->nb;
  const int64_t nf = int64_t(me->base) << L;
  const int64_t R = int64_t(k) * nf;
  m->uniform = false;
  for (int d = 0; d < 3; ++d) m->R[d] = R;
  const int64_t nc = int64_t(me->leaves.size()) / 4;
  m->n_cells = nc;
  if ((R + 1) * (R + 1) * (R + 1) >= (int64_t(1) << 62)) return fail(MF_EINVAL, "lattice too large");

  // local node offsets, x fastest
  std::vector<int> loc(3 * nb);
  for (int c = 0, i = 0; c <= k; ++c)
    for (int b = 0; b <= k; ++b)
      for (int a = 0; a <= k; ++a, ++i) { loc[3 * i] = a; loc[3 * i + 1] = b; loc[3 * i + 2] = c; }

  // every node of every leaf
  std::vector<int64_t> cell_keys(size_t(nc) * nb);
  m->cell_level.resize(nc);
  m->cell_anchor.resize(3 * nc);
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* lf = &me->leaves[4 * c];
    int lev = lf[0];
    int64_t step = int64_t(1) << (L - lev);
    m->cell_level[c] = uint8_t(lev);
    for (int d = 0; d < 3; ++d) m->cell_anchor[3 * c + d] = lf[1 + d];
    int64_t ax = lf[1] * k * step, ay = lf[2] * k * step, az = lf[3] * k * step;
    for (int i = 0; i < nb; ++i)
      cell_keys[c * nb + i] = key_of(ax + loc[3 * i] * step, ay + loc[3 * i + 1] * step, az + loc[3 * i + 2] * step, R);
  }
  std::vector<int64_t> pts(cell_keys);
  std::sort(pts.begin(), pts.end());
  pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
  const int64_t M = int64_t(pts.size());
  auto find_pt = [&](int64_t key) -> int64_t {
    auto it = std::lower_bound(pts.begin(), pts.end(), key);
    return (it != pts.end() && *it == key) ? int64_t(it - pts.begin()) : -1;
  };
  std::vector<int32_t> cell_pts(size_t(nc) * nb);
  for (size_t i = 0; i < cell_keys.size(); ++i) cell_pts[i] = int32_t(find_pt(cell_keys[i]));
  cell_keys.clear();
  cell_keys.shrink_to_fit();

  // 1D Lagrange values at half steps: lw[a][p] = l_a(p / 2k)
  std::vector<double> lw((k + 1) * (2 * k + 1));
  for (int a = 0; a <= k; ++a)
    for (int p = 0; p <= 2 * k; ++p) lw[a * (2 * k + 1) + p] = lagrange_at_half_step(k, a, p);

  // candidate half-step offsets on the closed cell boundary with an odd coordinate
  std::vector<int> cand;
  for (int r = 0; r <= 2 * k; ++r)
    for (int q = 0; q <= 2 * k; ++q)
      for (int p = 0; p <= 2 * k; ++p) {
        bool bnd = p == 0 || q == 0 || r == 0 || p == 2 * k || q == 2 * k || r == 2 * k;
        bool odd = (p & 1) || (q & 1) || (r & 1);
        if (bnd && odd) { cand.push_back(p); cand.push_back(q); cand.push_back(r); }
      }

  // direct interpolation rows of hanging points: point -> (master point, weight)
  std::unordered_map<int64_t, std::vector<std::pair<int64_t, double>>> direct;
  for (int64_t c = 0; c < nc; ++c) {
    int lev = m->cell_level[c];
    if (lev >= L) continue;
    int64_t step = int64_t(1) << (L - lev), hs = step / 2;
    int64_t ax = int64_t(m->cell_anchor[3 * c]) * k * step, ay = int64_t(m->cell_anchor[3 * c + 1]) * k * step,
            az = int64_t(m->cell_anchor[3 * c + 2]) * k * step;
    for (size_t t = 0; t < cand.size(); t += 3) {
      int p = cand[t], q = cand[t + 1], r = cand[t + 2];
      int64_t pi = find_pt(key_of(ax + p * hs, ay + q * hs, az + r * hs, R));
      if (pi < 0) continue;
      std::vector<std::pair<int64_t, double>> w;
      for (int i = 0; i < nb; ++i) {
        double v = lw[loc[3 * i] * (2 * k + 1) + p] * lw[loc[3 * i + 1] * (2 * k + 1) + q] * lw[loc[3 * i + 2] * (2 * k + 1) + r];
        if (v != 0.0) w.emplace_back(cell_pts[c * nb + i], v);
      }
      auto it = direct.find(pi);
      if (it == direct.end()) direct.emplace(pi, std::move(w));
      else {
        // another coarse leaf sharing the point must interpolate identically
        auto a = it->second, b = w;
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        if (a != b) return fail(MF_EINVAL, "inconsistent hanging-node interpolation (mesh not 2:1?)");
      }
    }
  }

  // free numbering in key order
  std::vector<int64_t> free_of(M, -1), hang_of(M, -1);
  int64_t nfree = 0, nhang = 0;
  for (int64_t p = 0; p < M; ++p) {
    if (direct.count(p)) hang_of[p] = nhang++;
    else free_of[p] = nfree++;
  }
  if (nfree >= (int64_t(1) << 31)) return fail(MF_EINVAL, "octree map exceeds 2^31 DoFs");
  m->n_dofs = nfree;
  m->free_keys.resize(nfree);
  for (int64_t p = 0; p < M; ++p)
    if (free_of[p] >= 0) m->free_keys[free_of[p]] = pts[p];

  // resolve chains to free masters (memoised), sum equal masters, drop exact zeros
  std::unordered_map<int64_t, std::map<int64_t, double>> resolved;
  std::function<const std::map<int64_t, double>&(int64_t, int)> resolve =
      [&](int64_t p, int depth) -> const std::map<int64_t, double>& {
    auto it = resolved.find(p);
    if (it != resolved.end()) return it->second;
    std::map<int64_t, double> out;
    if (depth < 64) {
      for (auto& mw : direct[p]) {
        if (direct.count(mw.first)) {
          const auto& sub = resolve(mw.first, depth + 1);
          for (auto& s : sub) out[s.first] += mw.second * s.second;
        } else {
          out[free_of[mw.first]] += mw.second;
        }
      }
    }
    for (auto i2 = out.begin(); i2 != out.end();) i2 = (i2->second == 0.0) ? out.erase(i2) : std::next(i2);
    return resolved.emplace(p, std::move(out)).first->second;
  };
  m->con_rowptr.assign(1, 0);
  m->con_cols.clear();
  m->con_w.clear();
  std::vector<int64_t> hang_pts;
  hang_pts.reserve(nhang);
  for (int64_t p = 0; p < M; ++p)
    if (hang_of[p] >= 0) hang_pts.push_back(p);
  for (int64_t p : hang_pts) {
    const auto& row = resolve(p, 0);
    for (auto& s : row) {
      m->con_cols.push_back(int32_t(s.first));
      m->con_w.push_back(s.second);
    }
    m->con_rowptr.push_back(int64_t(m->con_cols.size()));
  }

  // cell map
  m->cell_map.resize(size_t(nc) * nb);
  for (size_t i = 0; i < m->cell_map.size(); ++i) {
    int64_t p = cell_pts[i];
    m->cell_map[i] = free_of[p] >= 0 ? int32_t(free_of[p]) : int32_t(-1 - hang_of[p]);
  }
  build_dirichlet_lists(m);
  return MF_OK;
}

mf_status upload_dofmap(mf_dofmap* m) {
  cudaStream_t s = m->mesh->ctx->stream;
  if (!m->dirichlet_list.empty()) MF_TRY(m->d_dir_list.upload(m->dirichlet_list, s));
  if (m->uniform) return MF_OK;
  const int64_t nc = m->n_cells, nb = m->nb;
  m->n_cells_pad = (nc + 31) / 32 * 32;
  // processing order: cells without constrained nodes first (uniform control flow)
  std::vector<int32_t> order, order_c;
  std::vector<uint8_t> flags(nc, 0);
  for (int64_t c = 0; c < nc; ++c) {
    bool con = false;
    for (int i = 0; i < nb; ++i) con |= m->cell_map[c * nb + i] < 0;
    flags[c] = con ? 1 : 0;
    (con ? order_c : order).push_back(int32_t(c));
  }
  m->n_unconstrained = int64_t(order.size());
  m->n_constrained_cells = int64_t(order_c.size());
  order.insert(order.end(), order_c.begin(), order_c.end());
  std::vector<int32_t> soa(size_t(m->n_cells_pad) * nb, 0);
  for (int64_t c = 0; c < nc; ++c)
    for (int i = 0; i < nb; ++i) soa[size_t(i) * m->n_cells_pad + c] = m->cell_map[c * nb + i];
  MF_TRY(m->d_cell_map.upload(soa, s));
  MF_TRY(m->d_cell_level.upload(m->cell_level, s));
  MF_TRY(m->d_cell_flags.upload(flags, s));
  MF_TRY(m->d_order.upload(order, s));
  std::vector<int32_t> rp(m->con_rowptr.begin(), m->con_rowptr.end());
  if (rp.empty()) rp.push_back(0);
  MF_TRY(m->d_con_rowptr.upload(rp, s));
  std::vector<float> wf(m->con_w.begin(), m->con_w.end());
  if (!m->con_cols.empty()) {
    MF_TRY(m->d_con_cols.upload(m->con_cols, s));
    MF_TRY(m->d_con_w.upload(m->con_w, s));
    MF_TRY(m->d_con_wf.upload(wf, s));
  }
  if (!m->dirichlet_list.empty()) MF_TRY(m->d_dir_flag.upload(m->dirichlet, s));
  MF_CUDA_TRY(cudaStreamSynchronize(s));
  return MF_OK;
}

}  // namespace mf
