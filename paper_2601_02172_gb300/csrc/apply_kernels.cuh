// Matrix-free stiffness apply of the scaled X-FEM system (eqs. Kapp, b, resVector):
//   q = sum_e Lambda_e^T int_e B~^T C (eps_bar + B~ d_e)        (eps_bar only in TOTAL mode)
// with fused reductions <d, A d> = sum_e int eps(d) : C : eps(d) and int_Y C (eps_bar + grad^s d).
//
// Uncut tets (constant strain, one phase): a 2.5-D marching kernel.  A block of kTZ x kTY
// (16 x 16) threads owns one voxel column each (y, z) and walks along x; node planes of d are
// staged in shared memory, each voxel's six Kuhn tets are evaluated once, the 8 corner forces are
// combined along z by warp shuffles and along y through shared memory, and the x direction is
// carried in registers, so every node force is written exactly once with a plain store.
//
// Cut tets: apply_cut.cuh (one thread per cut tet, atomics after the uncut kernel).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "xfft_kernels.h"

namespace xfft {

constexpr int kTZ = 16;  // threads along z (half a warp; a warp covers two y rows)
constexpr int kTY = 16;  // threads along y
#ifndef XFFT_UNCUT_CX
#define XFFT_UNCUT_CX 32
#endif
constexpr int kCX = XFFT_UNCUT_CX;  // output planes per block along x
#ifndef XFFT_UNCUT_MINB
#define XFFT_UNCUT_MINB 2  // resident blocks per SM asked of the FP32 uncut kernel
#endif
#ifndef XFFT_UNCUT_MINB64
#define XFFT_UNCUT_MINB64 2  // resident blocks per SM asked of the FP64 uncut kernel
#endif
#ifndef XFFT_UNCUT_MINBDW
#define XFFT_UNCUT_MINBDW 1  // resident blocks per SM asked of the double-word uncut kernel
#endif

template <typename T>
__device__ __forceinline__ T cut_real(const CutData& cd, int f, int e);
template <>
__device__ __forceinline__ double cut_real<double>(const CutData& cd, int f, int e) {
  return cd.dp[(long long)f * cd.ncut + e];
}
template <>
__device__ __forceinline__ float cut_real<float>(const CutData& cd, int f, int e) {
  return cd.fp[(long long)f * cd.ncut + e];
}
template <>
__device__ __forceinline__ dw cut_real<dw>(const CutData& cd, int f, int e) {
  return dw(cd.dp[(long long)f * cd.ncut + e]);
}

// symmetric tensor stored as (00, 11, 22, 12, 02, 01)
template <typename T>
__device__ __forceinline__ T sym_at(const T (&s)[6], int i, int j) {
  if (i == j) return s[i];
  const int k = i + j;  // 1 -> (0,1), 2 -> (0,2), 3 -> (1,2)
  return k == 1 ? s[5] : (k == 2 ? s[4] : s[3]);
}

template <typename T>
__device__ __forceinline__ void mandel_to_tensor(const double* e, T (&E)[6]) {
  const double r = 0.70710678118654752440;
  E[0] = (T)e[0];
  E[1] = (T)e[1];
  E[2] = (T)e[2];
  E[3] = (T)(e[3] * r);
  E[4] = (T)(e[4] * r);
  E[5] = (T)(e[5] * r);
}

template <typename T>
__device__ __forceinline__ void iso_stress(const T (&e)[6], T lam, T mu, T (&s)[6]) {
  const T tr = e[0] + e[1] + e[2];
  const T m2 = mu + mu;
  s[0] = lam * tr + m2 * e[0];
  s[1] = lam * tr + m2 * e[1];
  s[2] = lam * tr + m2 * e[2];
  s[3] = m2 * e[3];
  s[4] = m2 * e[4];
  s[5] = m2 * e[5];
}

template <typename T>
__device__ __forceinline__ T ddot(const T (&s)[6], const T (&e)[6]) {
  return s[0] * e[0] + s[1] * e[1] + s[2] * e[2] + T(2) * (s[3] * e[3] + s[4] * e[4] + s[5] * e[5]);
}

// One uncut Kuhn tet t of a voxel with corner displacements u: adds its corner forces to F and
// its energy/stress integrals to the accumulators.
template <typename T, int t, bool TOTAL>
__device__ __forceinline__ void tet_uncut(const T (&u)[8][3], T (&F)[8][3], unsigned code,
                                          const T (&lm)[kMaxPhases], const T (&mu2)[kMaxPhases],
                                          const T (&ih)[3],
                                          const T (&w)[3], T vol, const T (&E)[6], T& en,
                                          T (&sg)[6]) {
  constexpr int p = perm_p(t), q = perm_q(t), r = perm_r(t);
  constexpr int c1 = tet_c1(t), c2 = tet_c2(t);
  const unsigned cd = (code >> (2 * t)) & 3u;
  if (cd == kCodeCut) return;
  const T lam = lm[code_phase(cd)], mu = mu2[code_phase(cd)];
  T H[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    H[i][p] = (u[c1][i] - u[0][i]) * ih[p];
    H[i][q] = (u[c2][i] - u[c1][i]) * ih[q];
    H[i][r] = (u[7][i] - u[c2][i]) * ih[r];
  }
  T e[6];
  e[0] = H[0][0];
  e[1] = H[1][1];
  e[2] = H[2][2];
  e[3] = T(0.5) * (H[1][2] + H[2][1]);
  e[4] = T(0.5) * (H[0][2] + H[2][0]);
  e[5] = T(0.5) * (H[0][1] + H[1][0]);
  if (TOTAL) {
#pragma unroll
    for (int k = 0; k < 6; ++k) e[k] += E[k];
  }
  T s[6];
  iso_stress(e, lam, mu, s);
  en += vol * ddot(s, e);
  sg[0] += vol * s[0];
  sg[1] += vol * s[1];
  sg[2] += vol * s[2];
  sg[3] += vol * s[3];
  sg[4] += vol * s[4];
  sg[5] += vol * s[5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T tp = w[p] * sym_at(s, i, p);
    const T tq = w[q] * sym_at(s, i, q);
    const T tr = w[r] * sym_at(s, i, r);
    F[0][i] -= tp;
    F[c1][i] += tp - tq;
    F[c2][i] += tq - tr;
    F[7][i] += tr;
  }
}

// ---------------------------------------------------------------- uncut stencil
// Node values staged in shared memory as 4-vectors (one 16- or 32-byte load per corner).
template <typename T>
struct Node4 {
  T x, y, z, w;
};
template <typename T>
__device__ __forceinline__ T comp(const Node4<T>& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : v.z);
}

// Per-voxel coefficients of the uncut tets, per phase ph (one interface: 0 minus, 1 plus; NPH
// phases in all) and axis k:
//   lw[ph][k] = lambda w_k s_v, mw[ph][k] = mu w_k s_v with w_k = |T| / h_k^2 on a uniform grid
//   (raw node differences) or |T| / h_k otherwise (differences scaled by 1/h_k).
template <typename T, bool UNIFORM, int NPH>
struct Coef {
  T lw[NPH][UNIFORM ? 1 : 3];
  T mw[NPH][UNIFORM ? 1 : 3];
  __device__ __forceinline__ T l(int ph, int k) const { return lw[ph][UNIFORM ? 0 : k]; }
  __device__ __forceinline__ T m(int ph, int k) const { return mw[ph][UNIFORM ? 0 : k]; }
};

// One uncut Kuhn tet: the displacement-gradient columns of the tet are the node differences
// along its path 0 -> e_p -> e_p+e_q -> (1,1,1); the edge tensions T_k = w_k sigma e_k move
// the corner forces: F[0] -= T_p, F[c1] += T_p - T_q, F[c2] += T_q - T_r, F[7] += T_r.
// Edge tensions of a voxel, summed over its tets: first edges 0 -> e_p (TE0[p]), middle edges
// e_p -> e_p + e_q (TEM[p][q]), last edges e_p + e_q -> (1,1,1) (TEL[r], r the third axis).
template <typename T>
struct EdgeT {
  T e0[3][3], em[3][3][3], el[3][3];
};

// EDGE: add the tet's tensions to the voxel's edge sums (corner forces formed once per voxel by
// edge_forces); otherwise add them to the corner forces F directly.
template <typename T, int t, bool TOTAL, bool SIG, bool UNIFORM, int NPH, bool EDGE = false>
__device__ __forceinline__ void tet_stencil(const Node4<T> (&u)[8], T (&F)[8][3], unsigned code,
                                            const Coef<T, UNIFORM, NPH>& cf, const T (&ih)[3],
                                            const T (&hk)[3], const T (&Eb)[3][3], T& en, T (&sg)[6],
                                            EdgeT<T>* te = nullptr) {
  constexpr int p = perm_p(t), q = perm_q(t), r = perm_r(t);
  constexpr int c1 = tet_c1(t), c2 = tet_c2(t);
  const unsigned cd = (code >> (2 * t)) & 3u;
  if (cd == kCodeCut) return;
  const int ph = NPH == 2 ? (int)cd : code_phase(cd);
  T G[3][3];  // G[k][i]: column k (axis k) of the gradient, component i
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G[p][i] = comp(u[c1], i) - comp(u[0], i);
    G[q][i] = comp(u[c2], i) - comp(u[c1], i);
    G[r][i] = comp(u[7], i) - comp(u[c2], i);
  }
  if (!UNIFORM) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      G[0][i] *= ih[0];
      G[1][i] *= ih[1];
      G[2][i] *= ih[2];
    }
  }
  T Dr[3][3];  // unmodified columns for the energy
  if (SIG) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) Dr[k][i] = G[k][i];
  }
  if (TOTAL) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) G[k][i] += Eb[i][k];
  }
  const T tr = G[0][0] + G[1][1] + G[2][2];
  const T s01 = G[0][1] + G[1][0], s02 = G[0][2] + G[2][0], s12 = G[1][2] + G[2][1];
  T Tn[3][3];  // Tn[k][i] = tension on the column-k edge, component i
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T lw = cf.l(ph, k), mw = cf.m(ph, k);
    Tn[k][k] = lw * tr + (mw + mw) * G[k][k];
  }
  {
    Tn[0][1] = cf.m(ph, 0) * s01;
    Tn[1][0] = cf.m(ph, 1) * s01;
    Tn[0][2] = cf.m(ph, 0) * s02;
    Tn[2][0] = cf.m(ph, 2) * s02;
    Tn[1][2] = cf.m(ph, 1) * s12;
    Tn[2][1] = cf.m(ph, 2) * s12;
  }
  if (EDGE) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      te->e0[p][i] += Tn[p][i];
      te->em[p][q][i] += Tn[q][i];
      te->el[r][i] += Tn[r][i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      F[0][i] -= Tn[p][i];
      F[c1][i] += Tn[p][i] - Tn[q][i];
      F[c2][i] += Tn[q][i] - Tn[r][i];
      F[7][i] += Tn[r][i];
    }
  }
  if (SIG) {
    // |T| sigma_ik = h_k Tn[k][i]; |T| sigma : eps = sum_k hk[k] Tn[k] . Dr[k]
    sg[0] += hk[0] * Tn[0][0];
    sg[1] += hk[1] * Tn[1][1];
    sg[2] += hk[2] * Tn[2][2];
    sg[3] += hk[1] * Tn[1][2];
    sg[4] += hk[0] * Tn[0][2];
    sg[5] += hk[0] * Tn[0][1];
    T e = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      e += (UNIFORM ? T(1) : hk[k]) * (Tn[k][0] * Dr[k][0] + Tn[k][1] * Dr[k][1] + Tn[k][2] * Dr[k][2]);
    en += e;
  }
}

// Corner forces of a voxel from its edge tensions: each edge pulls its end corner and pushes
// its start corner (corner index bits: x = 1, y = 2, z = 4).
template <typename T>
__device__ __forceinline__ void edge_forces(const EdgeT<T>& te, T (&F)[8][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    F[0][i] = -(te.e0[0][i] + te.e0[1][i] + te.e0[2][i]);
    F[7][i] = te.el[0][i] + te.el[1][i] + te.el[2][i];
    F[1][i] = te.e0[0][i] - te.em[0][1][i] - te.em[0][2][i];
    F[2][i] = te.e0[1][i] - te.em[1][0][i] - te.em[1][2][i];
    F[4][i] = te.e0[2][i] - te.em[2][0][i] - te.em[2][1][i];
    F[3][i] = te.em[0][1][i] + te.em[1][0][i] - te.el[2][i];
    F[5][i] = te.em[0][2][i] + te.em[2][0][i] - te.el[1][i];
    F[6][i] = te.em[1][2][i] + te.em[2][1][i] - te.el[0][i];
  }
}

#ifndef XFFT_EDGE_FORCES
#define XFFT_EDGE_FORCES 1  // corner forces from per-voxel edge tension sums
#endif

template <typename T, bool TOTAL, bool SIG, bool UNIFORM, bool FUSED, int NPH>
__global__ void __launch_bounds__(kTZ* kTY, std::is_same<T, dw>::value     ? XFFT_UNCUT_MINBDW
                                             : sizeof(T) == 8 ? XFFT_UNCUT_MINB64
                                                              : XFFT_UNCUT_MINB)
    k_apply_uncut(const typename Store<T>::type* __restrict__ d, typename Store<T>::type* __restrict__ q,
                  const ApplyArgs a, int nxchunks) {
  typedef typename Store<T>::type S;
  const int tz = threadIdx.x, ty = threadIdx.y;
  const int tid = tz + kTZ * ty;
  const int rhs = blockIdx.z / nxchunks;
  const int xc = blockIdx.z - rhs * nxchunks;
  if (a.active && !a.active[rhs]) return;
  if (a.units_uncut && tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && xc == 0)
    atomicAdd(a.units_uncut, 1ULL);
  const GridDev& g = a.g;
  const int n0 = g.n0, n1 = g.n1, n2 = g.n2;
  const long long N = g.N;
  const long long plane = (long long)n1 * n2;
  const int z0 = blockIdx.x * (kTZ - 1), y0 = blockIdx.y * (kTY - 1), x0 = xc * kCX;
  const int x1 = min(x0 + kCX, n0);
  const S* dr = d + rhs * a.stride;
  S* qr = q + rhs * a.stride;

  __shared__ Node4<T> P[2][kTY + 1][kTZ + 1];
  __shared__ T Ys[2][3][kTY][kTZ];
  __shared__ double red[7 * 32];

  constexpr int kPlaneNodes = (kTY + 1) * (kTZ + 1);
  int ld_slot[2];
  long long ld_off[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int lin = tid + k * kTZ * kTY;
    ld_slot[k] = lin < kPlaneNodes ? lin : -1;
    const int iy = lin / (kTZ + 1), iz = lin - iy * (kTZ + 1);
    const int yy = ((y0 - 1 + iy) % n1 + n1) % n1;
    const int zz = ((z0 - 1 + iz) % n2 + n2) % n2;
    ld_off[k] = (long long)yy * n2 + zz;
  }
  const int yg = y0 - 1 + ty, zg = z0 - 1 + tz;
  const int yv = (yg % n1 + n1) % n1, zv = (zg % n2 + n2) % n2;
  const bool own = ty >= 1 && tz >= 1 && yg < n1 && zg < n2;

  T ih[3], hk[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ih[k] = (T)(1.0 / g.h[k]);
    hk[k] = (T)g.h[k];
  }
  // phase coefficients without the voxel scale (converted once; no FP64 work in the loop)
  T lw0[NPH][3], mw0[NPH][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double wk = UNIFORM ? g.vol_tet / (g.h[0] * g.h[0]) : g.vol_tet / g.h[k];
#pragma unroll
    for (int ph = 0; ph < NPH; ++ph) {
      lw0[ph][k] = (T)(a.ph.lam[ph] * wk);
      mw0[ph][k] = (T)(a.ph.mu[ph] * wk);
    }
  }
  T Eb[3][3] = {};
  if (TOTAL) {
    const double* e = a.eps + 6 * rhs;
    const double rs = 0.70710678118654752440;
    const double sc = UNIFORM ? g.h[0] : 1.0;  // raw differences carry a factor h
    Eb[0][0] = (T)(e[0] * sc);
    Eb[1][1] = (T)(e[1] * sc);
    Eb[2][2] = (T)(e[2] * sc);
    Eb[1][2] = Eb[2][1] = (T)(e[3] * rs * sc);
    Eb[0][2] = Eb[2][0] = (T)(e[4] * rs * sc);
    Eb[0][1] = Eb[1][0] = (T)(e[5] * rs * sc);
  }

  // fused CG update: the block owns the plane nodes with 1 <= iy <= kTY-1, 1 <= iz <= kTZ-1
  // inside the grid; it stores d_new and updates u there (other blocks only read them as halo)
  const S* zr = FUSED ? static_cast<const S*>(a.fz) + rhs * a.stride : nullptr;
  S* dnr = FUSED ? static_cast<S*>(a.fdnew) + rhs * a.stride : nullptr;
  S* ur = FUSED ? static_cast<S*>(a.fu) + rhs * a.stride : nullptr;
  const T fa = FUSED ? (T)a.st[rhs].alpha : T(0);
  const T fb = FUSED ? (T)a.st[rhs].beta : T(0);
  bool slot_own[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int lin = tid + k * kTZ * kTY;
    const int iy = lin / (kTZ + 1), iz = lin - iy * (kTZ + 1);
    slot_own[k] = ld_slot[k] >= 0 && iy >= 1 && iy <= kTY - 1 && iz >= 1 && iz <= kTZ - 1 &&
                  y0 - 1 + iy < n1 && z0 - 1 + iz < n2;
  }

  // Two-stage plane pipeline: fetch() issues the global loads of a node plane into registers,
  // commit() (one step later, after the arithmetic of the current step was issued) forms the
  // fused update, stores the block's own nodes and fills the shared-memory plane.
  T pf[2][9];  // per load slot: z (or d) 0..2, d_old 3..5, u 6..8
  long long pf_nd[2] = {0, 0};
  bool pf_own[2] = {false, false};
  auto fetch = [&](int xp, bool own_plane) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      pf_own[k] = false;
      if (ld_slot[k] >= 0) {
        const long long nd = (long long)xp * plane + ld_off[k];
        pf_nd[k] = nd;
        if (FUSED) {
          pf[k][0] = from_store<T>(zr[nd]);
          pf[k][1] = from_store<T>(zr[N + nd]);
          pf[k][2] = from_store<T>(zr[2 * N + nd]);
          pf[k][3] = from_store<T>(dr[nd]);
          pf[k][4] = from_store<T>(dr[N + nd]);
          pf[k][5] = from_store<T>(dr[2 * N + nd]);
          pf_own[k] = own_plane && slot_own[k];
          if (pf_own[k]) {
            pf[k][6] = from_store<T>(ur[nd]);
            pf[k][7] = from_store<T>(ur[N + nd]);
            pf[k][8] = from_store<T>(ur[2 * N + nd]);
          }
        } else {
          pf[k][0] = from_store<T>(dr[nd]);
          pf[k][1] = from_store<T>(dr[N + nd]);
          pf[k][2] = from_store<T>(dr[2 * N + nd]);
        }
      }
    }
  };
  auto commit = [&](int buf) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (ld_slot[k] >= 0) {
        const int iy = ld_slot[k] / (kTZ + 1), iz = ld_slot[k] - iy * (kTZ + 1);
        Node4<T> v;
        if (FUSED) {
          v.x = pf[k][0] + fb * pf[k][3];
          v.y = pf[k][1] + fb * pf[k][4];
          v.z = pf[k][2] + fb * pf[k][5];
          if (pf_own[k]) {
            const long long nd = pf_nd[k];
            dnr[nd] = to_store(v.x);
            dnr[N + nd] = to_store(v.y);
            dnr[2 * N + nd] = to_store(v.z);
            ur[nd] = to_store(pf[k][6] + fa * pf[k][3]);
            ur[N + nd] = to_store(pf[k][7] + fa * pf[k][4]);
            ur[2 * N + nd] = to_store(pf[k][8] + fa * pf[k][5]);
          }
        } else {
          v.x = pf[k][0];
          v.y = pf[k][1];
          v.z = pf[k][2];
        }
        v.w = T(0);
        P[buf][iy][iz] = v;
      }
    }
  };

  T pend[3] = {T(0), T(0), T(0)};
  T en = T(0);
  T sg[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  const int xfirst = ((x0 - 1) % n0 + n0) % n0;
  fetch(xfirst, false);
  commit(0);
  fetch(xfirst + 1 == n0 ? 0 : xfirst + 1, x0 < x1);
  // the voxel's phase code and modulus scale are loaded one x step ahead as well
  const long long yz = (long long)yv * n2 + zv;
  unsigned nx_code = a.code[(long long)xfirst * plane + yz];
  float nx_scale = a.scale ? a.scale[(long long)xfirst * plane + yz] : 1.0f;
  int xw = xfirst;  // the wrapped voxel index x0 - 1 + s, advanced without a division per step
  for (int s = 0; s <= x1 - x0; ++s, xw = xw + 1 >= n0 ? xw + 1 - n0 : xw + 1) {
    const unsigned code = nx_code;
    const T sv = from_store<T>(nx_scale);
    commit((s + 1) & 1);  // plane x0 + s
    if (s + 1 <= x1 - x0) {
      const int x1w = xw + 1 >= n0 ? xw + 1 - n0 : xw + 1;  // voxel of the next step
      const int xn = xw + 2 >= n0 ? xw + 2 - n0 : xw + 2;  // plane x0 + s + 1
      fetch(xn, x0 + s + 1 < x1);
      nx_code = a.code[(long long)x1w * plane + yz];
      if (a.scale) nx_scale = a.scale[(long long)x1w * plane + yz];
    }
    __syncthreads();
    Node4<T> u[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) u[c] = P[(s + (c & 1)) & 1][ty + ((c >> 1) & 1)][tz + ((c >> 2) & 1)];
    Coef<T, UNIFORM, NPH> cf;
#pragma unroll
    for (int ph = 0; ph < NPH; ++ph)
#pragma unroll
      for (int k = 0; k < (UNIFORM ? 1 : 3); ++k) {
        cf.lw[ph][k] = lw0[ph][k] * sv;
        cf.mw[ph][k] = mw0[ph][k] * sv;
      }
    T F[8][3];
    T ven = T(0);
    T vsg[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#if XFFT_EDGE_FORCES
    {
      EdgeT<T> te;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          te.e0[k][i] = te.el[k][i] = T(0);
#pragma unroll
          for (int l = 0; l < 3; ++l) te.em[k][l][i] = T(0);
        }
      tet_stencil<T, 0, TOTAL, SIG, UNIFORM, NPH, true>(u, F, code, cf, ih, hk, Eb, ven, vsg, &te);
      tet_stencil<T, 1, TOTAL, SIG, UNIFORM, NPH, true>(u, F, code, cf, ih, hk, Eb, ven, vsg, &te);
      tet_stencil<T, 2, TOTAL, SIG, UNIFORM, NPH, true>(u, F, code, cf, ih, hk, Eb, ven, vsg, &te);
      tet_stencil<T, 3, TOTAL, SIG, UNIFORM, NPH, true>(u, F, code, cf, ih, hk, Eb, ven, vsg, &te);
      tet_stencil<T, 4, TOTAL, SIG, UNIFORM, NPH, true>(u, F, code, cf, ih, hk, Eb, ven, vsg, &te);
      tet_stencil<T, 5, TOTAL, SIG, UNIFORM, NPH, true>(u, F, code, cf, ih, hk, Eb, ven, vsg, &te);
      edge_forces(te, F);
    }
#else
#pragma unroll
    for (int c = 0; c < 8; ++c) F[c][0] = F[c][1] = F[c][2] = T(0);
    tet_stencil<T, 0, TOTAL, SIG, UNIFORM, NPH>(u, F, code, cf, ih, hk, Eb, ven, vsg);
    tet_stencil<T, 1, TOTAL, SIG, UNIFORM, NPH>(u, F, code, cf, ih, hk, Eb, ven, vsg);
    tet_stencil<T, 2, TOTAL, SIG, UNIFORM, NPH>(u, F, code, cf, ih, hk, Eb, ven, vsg);
    tet_stencil<T, 3, TOTAL, SIG, UNIFORM, NPH>(u, F, code, cf, ih, hk, Eb, ven, vsg);
    tet_stencil<T, 4, TOTAL, SIG, UNIFORM, NPH>(u, F, code, cf, ih, hk, Eb, ven, vsg);
    tet_stencil<T, 5, TOTAL, SIG, UNIFORM, NPH>(u, F, code, cf, ih, hk, Eb, ven, vsg);
#endif
    if (SIG && own && s >= 1) {
      en += ven;
#pragma unroll
      for (int k = 0; k < 6; ++k) sg[k] += vsg[k];
    }
    T G2[2][2][3];
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const T up = shfl_up_t<T>(0xffffffffu, F[dx + 2 * dy + 4][i], 1, kTZ);
          G2[dx][dy][i] = F[dx + 2 * dy][i] + up;
        }
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
      for (int i = 0; i < 3; ++i) Ys[dx][i][ty][tz] = G2[dx][1][i];
    __syncthreads();
    if (own) {
      T H0[3], H1[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        H0[i] = G2[0][0][i] + Ys[0][i][ty - 1][tz];
        H1[i] = G2[1][0][i] + Ys[1][i][ty - 1][tz];
      }
      if (s >= 1) {
        const long long nd = (long long)xw * plane + (long long)yv * n2 + zv;
        const T q0 = pend[0] + H0[0], q1 = pend[1] + H0[1], q2 = pend[2] + H0[2];
        qr[nd] = to_store(q0);
        qr[N + nd] = to_store(q1);
        qr[2 * N + nd] = to_store(q2);
        if (!SIG) en += q0 * u[0].x + q1 * u[0].y + q2 * u[0].z;  // <d, q> of this node
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) pend[i] = H1[i];
    }
  }
  const double r2 = 1.41421356237309504880;
  double v[7] = {to_double(en), to_double(sg[0]), to_double(sg[1]), to_double(sg[2]),
                 to_double(sg[3]) * r2, to_double(sg[4]) * r2, to_double(sg[5]) * r2};
  double tot[7];
  block_sum<7>(v, red, tot);
  if (tid == 0) {
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * xc);
#pragma unroll
    for (int k = 0; k < 7; ++k) a.partials[((long long)rhs * 7 + k) * a.nparts + bid] = tot[k];
  }
}

// Stencil launches of one phase count NPH (2: one interface; 3: two interfaces).  The phase
// counts are instantiated in separate translation units (apply.cu, apply_multi.cu).
template <typename T, int NPH>
cudaError_t launch_uncut_nph(const typename Store<T>::type* d, typename Store<T>::type* q,
                             const ApplyArgs& a, int n_rhs, cudaStream_t s) {
  const GridDev& g = a.g;
  const int gz = (g.n2 + kTZ - 2) / (kTZ - 1);
  const int gy = (g.n1 + kTY - 2) / (kTY - 1);
  const int gx = (g.n0 + kCX - 1) / kCX;
  dim3 block(kTZ, kTY, 1);
  dim3 grid(gz, gy, gx * n_rhs);
  const bool uni = g.h[0] == g.h[1] && g.h[1] == g.h[2];
  const bool sig = a.want_sig || a.eps;
#define XFFT_LAUNCH(TOT, SG, UNI) k_apply_uncut<T, TOT, SG, UNI, false, NPH><<<grid, block, 0, s>>>(d, q, a, gx)
#define XFFT_LAUNCH_F(SG, UNI) k_apply_uncut<T, false, SG, UNI, true, NPH><<<grid, block, 0, s>>>(d, q, a, gx)
  if (a.fz) {
    // the fused CG update serves the FP32 and FP64 solvers (not the double-word residuals)
    if constexpr (!std::is_same<T, dw>::value) {
      if (sig) {
        if (uni) XFFT_LAUNCH_F(true, true);
        else XFFT_LAUNCH_F(true, false);
      } else {
        if (uni) XFFT_LAUNCH_F(false, true);
        else XFFT_LAUNCH_F(false, false);
      }
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (a.eps) {
    if (uni) XFFT_LAUNCH(true, true, true);
    else XFFT_LAUNCH(true, true, false);
  } else if (sig) {
    if (uni) XFFT_LAUNCH(false, true, true);
    else XFFT_LAUNCH(false, true, false);
  } else {
    if (uni) XFFT_LAUNCH(false, false, true);
    else XFFT_LAUNCH(false, false, false);
  }
#undef XFFT_LAUNCH
#undef XFFT_LAUNCH_F
  return cudaGetLastError();
}

#define XFFT_APPLY_INST_NPH(EXT, T, NPH)                                                         \
  EXT template cudaError_t launch_uncut_nph<T, NPH>(const Store<T>::type*, Store<T>::type*,      \
                                                    const ApplyArgs&, int, cudaStream_t);

}  // namespace xfft
