// fv_host.cpp -- cold path of fv_mesh_load: validation, Morton renumbering,
// face extraction through node->tet adjacency, FP64 geometry and
// least-squares weights.  Compiled with -ffp-contract=off so the geometry is
// exactly what the formulas below say (the local time step and therefore
// the temporal levels depend on it bit for bit).
//
// Sec. 2.1 of the paper: the solver manipulates cells and faces; fields live
// on cells and fluxes on faces.  Conventions:
//  - face j of a tet is the face opposite its local node j;
//  - a face is owned by the tet with the smaller index in the caller's
//    order; its unit normal points out of the owner;
//  - the area vector is 1/2 (q1 - q0) x (q2 - q0) over the owner's face nodes
//    in ascending local order, flipped to point away from the opposite node;
//  - on a boundary face, x_R is the mirror image of the owner's centroid in
//    the face plane (the ghost cell).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "fv_internal.h"

namespace {

template <typename Fn>
void parallel_for(int64_t n, Fn fn) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::min<int64_t>(hw ? hw : 1, std::max<int64_t>(1, n / 4096));
  nt = std::max(1, std::min(nt, 64));
  if (nt == 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=] { fn(a, b); });
  }
  for (auto &x : th) x.join();
}

inline void sub3(const double *a, const double *b, double *o) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
inline void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double *a, const double *b) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

// spread the low 21 bits of v to every third bit
inline uint64_t spread3(uint64_t v) {
  v &= 0x1fffff;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

}  // namespace

int fv_host_build(const double *xyz, int64_t n_nodes, const int64_t *tets, int64_t n_tets,
                  const int8_t *face_bc, HostMesh &H, std::string *err) {
  if (n_tets <= 0 || n_nodes <= 0 || n_tets > (int64_t)0x7fffffff / 16) {
    *err = "fv_mesh_load: bad sizes";
    return FV_ERR_INVALID_ARG;
  }
  const int64_t N = n_tets;
  // ---- validation, volumes and centroids in the caller's order
  std::vector<double> vol0(N), xc0(3 * N);
  std::atomic<int> bad{0};
  parallel_for(N, [&](int64_t a, int64_t b) {
    for (int64_t t = a; t < b; ++t) {
      const double *x[4];
      for (int v = 0; v < 4; ++v) {
        int64_t nd = tets[4 * t + v];
        if (nd < 0 || nd >= n_nodes) {
          bad = 1;
          return;
        }
        x[v] = xyz + 3 * nd;
      }
      double e1[3], e2[3], e3[3], c[3];
      sub3(x[1], x[0], e1);
      sub3(x[2], x[0], e2);
      sub3(x[3], x[0], e3);
      cross3(e1, e2, c);
      double V = dot3(c, e3) / 6.0;
      if (!(V > 0.0) || !std::isfinite(V)) bad = 2;
      vol0[t] = V;
      for (int d = 0; d < 3; ++d) xc0[3 * t + d] = (((x[0][d] + x[1][d]) + x[2][d]) + x[3][d]) * 0.25;
      for (int j = 0; j < 4; ++j) {
        int8_t bc = face_bc[4 * t + j];
        if (bc < 0 || bc > 2) bad = 3;
      }
    }
  });
  if (bad) {
    *err = bad == 1 ? "fv_mesh_load: node index out of range"
           : bad == 2 ? "fv_mesh_load: tet with non-positive volume (inverted or degenerate)"
                      : "fv_mesh_load: face_bc entry outside {0,1,2}";
    return bad == 1 || bad == 3 ? FV_ERR_INVALID_ARG : FV_ERR_BAD_MESH;
  }

  // ---- Morton order of the centroids (ties by caller's index)
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t t = 0; t < N; ++t)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], xc0[3 * t + d]);
      hi[d] = std::max(hi[d], xc0[3 * t + d]);
    }
  std::vector<std::pair<uint64_t, int64_t>> key(N);
  parallel_for(N, [&](int64_t a, int64_t b) {
    for (int64_t t = a; t < b; ++t) {
      uint64_t code = 0;
      for (int d = 0; d < 3; ++d) {
        double span = hi[d] - lo[d];
        double q = span > 0 ? (xc0[3 * t + d] - lo[d]) / span : 0.0;
        uint64_t iq = (uint64_t)std::min(2097151.0, std::max(0.0, q * 2097151.0));
        code |= spread3(iq) << d;
      }
      key[t] = {code, t};
    }
  });
  std::sort(key.begin(), key.end());
  H.N = N;
  H.new2old.resize(N);
  H.old2new.resize(N);
  for (int64_t i = 0; i < N; ++i) {
    H.new2old[i] = key[i].second;
    H.old2new[key[i].second] = i;
  }
  key.clear();
  key.shrink_to_fit();

  // ---- node -> tet adjacency (caller's tet indices)
  std::vector<int64_t> nstart(n_nodes + 1, 0);
  for (int64_t t = 0; t < N; ++t)
    for (int v = 0; v < 4; ++v) nstart[tets[4 * t + v] + 1]++;
  for (int64_t n = 0; n < n_nodes; ++n) nstart[n + 1] += nstart[n];
  std::vector<int64_t> ntet(4 * N), fillp(nstart.begin(), nstart.end() - 1);
  for (int64_t t = 0; t < N; ++t)
    for (int v = 0; v < 4; ++v) ntet[fillp[tets[4 * t + v]]++] = t;
  fillp.clear();

  // ---- face matching: the other tet sharing the three nodes of face j
  // nbr_old[4t+j] = caller index of the neighbour, or -1 on the boundary
  std::vector<int64_t> nbr_old(4 * N);
  std::vector<int8_t> nbr_j(4 * N);
  parallel_for(N, [&](int64_t a, int64_t b) {
    for (int64_t t = a; t < b; ++t)
      for (int j = 0; j < 4; ++j) {
        int64_t q[3];
        int m = 0;
        for (int v = 0; v < 4; ++v)
          if (v != j) q[m++] = tets[4 * t + v];
        int64_t n0 = q[0];
        if (nstart[q[1] + 1] - nstart[q[1]] < nstart[n0 + 1] - nstart[n0]) n0 = q[1];
        if (nstart[q[2] + 1] - nstart[q[2]] < nstart[n0 + 1] - nstart[n0]) n0 = q[2];
        int64_t found = -1;
        int fj = -1, count = 0;
        for (int64_t p = nstart[n0]; p < nstart[n0 + 1]; ++p) {
          int64_t u = ntet[p];
          if (u == t) continue;
          int hit = 0, miss = -1;
          for (int v = 0; v < 4; ++v) {
            int64_t x = tets[4 * u + v];
            if (x == q[0] || x == q[1] || x == q[2])
              ++hit;
            else
              miss = v;
          }
          if (hit == 3) {
            found = u;
            fj = miss;
            ++count;
          }
        }
        if (count > 1) bad = 4;
        nbr_old[4 * t + j] = found;
        nbr_j[4 * t + j] = (int8_t)fj;
        int8_t bc = face_bc[4 * t + j];
        if (found >= 0 && bc != FV_BC_INTERIOR) bad = 5;
        if (found < 0 && bc == FV_BC_INTERIOR) bad = 6;
      }
  });
  ntet.clear();
  ntet.shrink_to_fit();
  if (bad) {
    *err = bad == 4 ? "fv_mesh_load: non-manifold face (shared by more than two tets)"
           : bad == 5 ? "fv_mesh_load: interior face carries a boundary tag"
                      : "fv_mesh_load: boundary face without a wall/transmissive tag";
    return FV_ERR_BAD_MESH;
  }

  // ---- face numbering: owner-major in the new order, local j ascending
  std::vector<int> owned(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) {
    int64_t t = H.new2old[i];
    int c = 0;
    for (int j = 0; j < 4; ++j) {
      int64_t u = nbr_old[4 * t + j];
      if (u < 0 || t < u) ++c;
    }
    owned[i + 1] = owned[i] + c;
  }
  const int64_t F = owned[N];
  H.F = F;
  H.vol.resize(N);
  H.xc.resize(3 * N);
  H.cf.assign(4 * N, -1);
  H.cnb.assign(4 * N, 0);
  H.cown.assign(N, 0);
  H.fown.resize(F);
  H.fnb.resize(F);
  H.fn.resize(3 * F);
  H.farea.resize(F);
  H.fr.resize(3 * F);
  for (int64_t i = 0; i < N; ++i) {
    int64_t t = H.new2old[i];
    H.vol[i] = vol0[t];
    for (int d = 0; d < 3; ++d) H.xc[d * N + i] = xc0[3 * t + d];
  }
  parallel_for(N, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      int64_t t = H.new2old[i];
      int f = owned[i];
      for (int j = 0; j < 4; ++j) {
        int64_t u = nbr_old[4 * t + j];
        if (u >= 0 && u < t) continue;  // owned by the neighbour
        // this cell owns face f
        H.fown[f] = (int)i;
        H.cf[j * N + i] = f;
        H.cown[i] |= (uint8_t)(1u << j);
        if (u >= 0) {
          int64_t iu = H.old2new[u];
          int ju = nbr_j[4 * t + j];
          H.fnb[f] = (int)iu;
          H.cf[ju * N + iu] = f;
          H.cnb[j * N + i] = (int)iu;
          H.cnb[ju * N + iu] = (int)i;
        } else {
          int bc = face_bc[4 * t + j];
          H.fnb[f] = -bc;
          H.cnb[j * N + i] = -bc;
        }
        // geometry of the owner's local face j
        const double *q[3];
        int m = 0;
        for (int v = 0; v < 4; ++v)
          if (v != j) q[m++] = xyz + 3 * tets[4 * t + v];
        const double *xo = xyz + 3 * tets[4 * t + j];
        double e1[3], e2[3], av[3], to[3];
        sub3(q[1], q[0], e1);
        sub3(q[2], q[0], e2);
        cross3(e1, e2, av);
        for (int d = 0; d < 3; ++d) av[d] *= 0.5;
        sub3(xo, q[0], to);
        if (dot3(av, to) > 0.0)
          for (int d = 0; d < 3; ++d) av[d] = -av[d];
        double A = std::sqrt(dot3(av, av));
        double n[3] = {av[0] / A, av[1] / A, av[2] / A};
        H.farea[f] = A;
        for (int d = 0; d < 3; ++d) H.fn[d * F + f] = n[d];
        const double *xl = &xc0[3 * t];
        if (u >= 0) {
          const double *xr = &xc0[3 * u];
          for (int d = 0; d < 3; ++d) H.fr[d * F + f] = xr[d] - xl[d];
        } else {
          double xf[3], dl[3];
          for (int d = 0; d < 3; ++d) xf[d] = ((q[0][d] + q[1][d]) + q[2][d]) / 3.0;
          sub3(xf, xl, dl);
          double s = 2.0 * dot3(dl, n);
          for (int d = 0; d < 3; ++d) H.fr[d * F + f] = s * n[d];
        }
        ++f;
      }
    }
  });

  // ---- least-squares weights w_j = M^-1 r_j, M = sum_j r_j r_j^T
  H.lsw.resize(12 * N);
  parallel_for(N, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      double r[4][3];
      for (int j = 0; j < 4; ++j) {
        int f = H.cf[j * N + i];
        double s = (H.cown[i] >> j) & 1 ? 1.0 : -1.0;
        for (int d = 0; d < 3; ++d) r[j][d] = s * H.fr[d * F + f];
      }
      double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int j = 0; j < 4; ++j)
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) M[p][q] += r[j][p] * r[j][q];
      double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
      double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
      double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
      double det = (M[0][0] * c00 + M[0][1] * c01) + M[0][2] * c02;
      double inv[3][3];
      inv[0][0] = c00 / det;
      inv[1][0] = c01 / det;
      inv[2][0] = c02 / det;
      inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
      inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
      inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
      inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
      inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
      inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
      for (int j = 0; j < 4; ++j)
        for (int p = 0; p < 3; ++p)
          H.lsw[(3 * j + p) * N + i] = (inv[p][0] * r[j][0] + inv[p][1] * r[j][1]) + inv[p][2] * r[j][2];
    }
  });
  return FV_OK;
}
