// Cut-tet part of the matrix-free stiffness apply (eqs. Kapp, resVector on the elements that the
// interface crosses, Sec. 3 sub-tetrahedron integration).
//
// On side s of a cut tet the strain is linear in the parent P1 functions,
//   eps(x) = sum_b N_b(x) E_b,   E_b = es + c_b ew + sym(w_b (x) gamma),
// with es, ew the (constant) symmetric gradients of the standard and of the unscaled enriched
// vertex values u_b, w_b, c_b = |L_b| - s L_b and gamma = sum_b c_b grad N_b (the modified abs
// enrichment restricted to the side).  With the side moments m_b = int N_b, M_ab = int N_a N_b
// and P_b = sum_c M_bc c_c every integral is exact, and by linearity of the stress C(.):
//   std force   q_a  = sigma_bar g_a,          sigma_bar = C(V es + (m.c) ew + sym(W_m (x) gamma))
//   enr force   q~_a = T g_a + R_a gamma,      T = C((m.c) es + (c.M.c) ew + sym(W_P (x) gamma))
//               R_a gamma = m_a C(es) gamma + P_a C(ew) gamma + (lam + mu)(W_a . gamma) gamma
//                           + mu |gamma|^2 W_a
// with W_a = sum_b M_ab w_b, W_m = sum_a W_a, W_P = sum_b P_b w_b, g_a = grad N_a and V the side
// volume (sum_b P_b = m.c).  The geometry-only factors come from a per-tet record built at
// setup (setup.cu, k_cut_records); the tet's Kuhn type t is a compile-time constant of the body,
// so the gradients g_a = -e_p/h_p, e_p/h_p - e_q/h_q, e_q/h_q - e_r/h_r, e_r/h_r enter as sparse
// column differences.  The cut-tet list is grouped by tet type, so a warp runs one body.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "apply_kernels.cuh"
#include "xfft_kernels.h"

namespace xfft {

constexpr int kCutThreads = 128;
constexpr int kCutMaxR = 8;  // right-hand sides per launch (more are split over launches)
#ifndef XFFT_CUT_MINB
#define XFFT_CUT_MINB 4  // resident blocks per SM asked of the FP32 cut kernel
#endif

// Staging: the FP32 and FP64 kernels stage; the double-word kernel (one or two resident blocks
// per SM, long per-thread work) reads its records from global memory instead, where a block-wide
// barrier per group of tets would idle the SM.
template <typename T>
constexpr bool cut_staged() {
  return !std::is_same<T, dw>::value;
}

// Records are staged per block in shared memory, RecStride<S> reals apart: 68 floats (272 B)
// or 70 doubles (560 B), so that the 16-byte loads of 8 consecutive lanes hit distinct banks.
template <typename S>
struct RecStride;
template <>
struct RecStride<float> {
  static constexpr int v = kRec;
};
template <>
struct RecStride<double> {
  static constexpr int v = kRec + 2;
};
template <typename T>
constexpr size_t cut_smem_bytes() {
  typedef typename Store<T>::type S;
  return cut_staged<T>() ? (size_t)kCutThreads * RecStride<S>::v * sizeof(S) : 0;
}

// record loads from shared or global memory: 4 consecutive reals (16-byte aligned groups)
__device__ __forceinline__ void ld_rec4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void ld_rec4(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}
template <int n4, typename T, typename R>
__device__ __forceinline__ void ld_rec(const R* p, T* o) {
#pragma unroll
  for (int k = 0; k < n4; ++k) {
    R v[4];
    ld_rec4(p + 4 * k, v);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[4 * k + j] = from_store<T>(v[j]);
  }
}

template <typename T>
__device__ __forceinline__ void iso_C(const T (&e)[6], T lam, T mu, T (&s)[6]) {
  const T tr = e[0] + e[1] + e[2];
  const T m2 = mu + mu;
  const T lt = lam * tr;
  s[0] = lt + m2 * e[0];
  s[1] = lt + m2 * e[1];
  s[2] = lt + m2 * e[2];
  s[3] = m2 * e[3];
  s[4] = m2 * e[4];
  s[5] = m2 * e[5];
}

// (sym 3x3 stored as 00, 11, 22, 12, 02, 01) times a 3-vector
template <typename T>
__device__ __forceinline__ void symv(const T (&s)[6], const T (&v)[3], T (&o)[3]) {
  o[0] = s[0] * v[0] + s[5] * v[1] + s[4] * v[2];
  o[1] = s[5] * v[0] + s[1] * v[1] + s[3] * v[2];
  o[2] = s[4] * v[0] + s[3] * v[1] + s[2] * v[2];
}

// column k of a symmetric tensor
template <int k, typename T>
__device__ __forceinline__ T scol(const T (&s)[6], int i) {
  return i == k ? s[i] : (i + k == 1 ? s[5] : (i + k == 2 ? s[4] : s[3]));
}

// F_a += S g_a for the four vertices of Kuhn tet t (g_a sparse, see the file header)
template <int t, typename T>
__device__ __forceinline__ void add_forces(const T (&S)[6], const T (&ih)[3], T (&F)[4][3]) {
  constexpr int p = perm_p(t), q = perm_q(t), r = perm_r(t);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T cp = scol<p>(S, i) * ih[p];
    const T cq = scol<q>(S, i) * ih[q];
    const T cr = scol<r>(S, i) * ih[r];
    F[0][i] -= cp;
    F[1][i] += cp - cq;
    F[2][i] += cq - cr;
    F[3][i] += cr;
  }
}

// symmetric gradient of the vertex values v_a (a = 0..3) of Kuhn tet t
template <int t, typename T>
__device__ __forceinline__ void sym_grad(const T (&v)[4][3], const T (&ih)[3], T (&e)[6]) {
  constexpr int p = perm_p(t), q = perm_q(t), r = perm_r(t);
  T H[3][3];  // H[k][i] = d v_i / d x_k
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    H[p][i] = (v[1][i] - v[0][i]) * ih[p];
    H[q][i] = (v[2][i] - v[1][i]) * ih[q];
    H[r][i] = (v[3][i] - v[2][i]) * ih[r];
  }
  e[0] = H[0][0];
  e[1] = H[1][1];
  e[2] = H[2][2];
  e[3] = T(0.5) * (H[2][1] + H[1][2]);
  e[4] = T(0.5) * (H[2][0] + H[0][2]);
  e[5] = T(0.5) * (H[1][0] + H[0][1]);
}

// The same two operations with the gradients as data (Kuhn type known at run time only): the
// double-word kernel runs this single body, whatever the order of the tet types in its warps.
template <typename T>
struct TetGrad {
  T g[4][3];
};
template <typename T>
__device__ __forceinline__ void add_forces_rt(const T (&S)[6], const TetGrad<T>& G, T (&F)[4][3]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T v[3];
    symv(S, G.g[a], v);
#pragma unroll
    for (int i = 0; i < 3; ++i) F[a][i] += v[i];
  }
}
template <typename T>
__device__ __forceinline__ void sym_grad_rt(const T (&v)[4][3], const TetGrad<T>& G, T (&e)[6]) {
  T H[3][3];  // H[k][i] = d v_i / d x_k
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      H[k][i] = v[0][i] * G.g[0][k] + v[1][i] * G.g[1][k] + v[2][i] * G.g[2][k] + v[3][i] * G.g[3][k];
  e[0] = H[0][0];
  e[1] = H[1][1];
  e[2] = H[2][2];
  e[3] = T(0.5) * (H[2][1] + H[1][2]);
  e[4] = T(0.5) * (H[2][0] + H[0][2]);
  e[5] = T(0.5) * (H[1][0] + H[0][1]);
}

// the gradient operations of a cut-tet body: compile-time Kuhn type t (sparse) or, with t < 0,
// the run-time gradients G
template <int t, typename T>
__device__ __forceinline__ void forces_of(const T (&S)[6], const T (&ih)[3], const TetGrad<T>& G, T (&F)[4][3]) {
  if constexpr (t >= 0) add_forces<t>(S, ih, F);
  else add_forces_rt(S, G, F);
}
template <int t, typename T>
__device__ __forceinline__ void strain_of(const T (&v)[4][3], const T (&ih)[3], const TetGrad<T>& G, T (&e)[6]) {
  if constexpr (t >= 0) sym_grad<t>(v, ih, e);
  else sym_grad_rt(v, G, e);
}

// a * e1 + b * e2 + sym(W (x) g)
template <typename T>
__device__ __forceinline__ void strain_comb(T a, const T (&e1)[6], T b, const T (&e2)[6], const T (&W)[3],
                                            const T (&g)[3], T (&o)[6]) {
  o[0] = a * e1[0] + b * e2[0] + W[0] * g[0];
  o[1] = a * e1[1] + b * e2[1] + W[1] * g[1];
  o[2] = a * e1[2] + b * e2[2] + W[2] * g[2];
  o[3] = a * e1[3] + b * e2[3] + T(0.5) * (W[1] * g[2] + W[2] * g[1]);
  o[4] = a * e1[4] + b * e2[4] + T(0.5) * (W[0] * g[2] + W[2] * g[0]);
  o[5] = a * e1[5] + b * e2[5] + T(0.5) * (W[0] * g[1] + W[1] * g[0]);
}

// One side of one cut tet for one right-hand side: adds the side's forces to qs (standard) and
// qe (enriched, unscaled), its share of <d, q> to en (d's standard strain ed: sum_a u_a . q_a =
// sigma_bar : ed, sum_a w_a . q~_a = T : ew + sum_a w_a . R_a gamma) and, when SIG, its int sigma
// to sg.
template <int t, bool SIG, typename T, typename R>
__device__ __forceinline__ void cut_side(const R* __restrict__ S, const T (&ws)[4][3], const T (&es)[6],
                                         const T (&ed)[6], const T (&ew)[6], const T (&ih)[3],
                                         const TetGrad<T>& G, T (&qs)[4][3], T (&qe)[4][3], T& en,
                                         T (&sg)[6]) {
  T M[10], m[4], P[4], gx[8], sc[4];
  {
    T buf[28];
    ld_rec<7, T>(S, buf);
#pragma unroll
    for (int k = 0; k < 10; ++k) M[k] = buf[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      m[k] = buf[10 + k];
      P[k] = buf[14 + k];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) gx[k] = buf[18 + k];  // gamma (3), lambda, mu
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = buf[23 + k];  // V, m.c, c.M.c
  }
  const T gam[3] = {gx[0], gx[1], gx[2]};
  const T lam = gx[3], mu = gx[4];
  // W_a = sum_b M_ab w_b
  T W[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int x = 0; x < 3; ++x)
      W[a][x] = M[midx(a, 0)] * ws[0][x] + M[midx(a, 1)] * ws[1][x] + M[midx(a, 2)] * ws[2][x] +
                M[midx(a, 3)] * ws[3][x];
  T Wm[3], Wp[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    Wm[x] = (W[0][x] + W[1][x]) + (W[2][x] + W[3][x]);
    Wp[x] = P[0] * ws[0][x] + P[1] * ws[1][x] + P[2] * ws[2][x] + P[3] * ws[3][x];
  }
  // standard forces and the side's stress integral
  {
    T e[6], s[6];
    strain_comb(sc[0], es, sc[1], ew, Wm, gam, e);
    iso_C(e, lam, mu, s);
    forces_of<t>(s, ih, G, qs);
    en += ddot(s, ed);
    if (SIG) {
#pragma unroll
      for (int k = 0; k < 6; ++k) sg[k] += s[k];
    }
  }
  // enriched forces, T g_a
  {
    T e[6], s[6];
    strain_comb(sc[1], es, sc[2], ew, Wp, gam, e);
    iso_C(e, lam, mu, s);
    forces_of<t>(s, ih, G, qe);
    en += ddot(s, ew);
  }
  // enriched forces, R_a gamma
  T v1[3], v2[3];
  {
    T s[6];
    iso_C(es, lam, mu, s);
    symv(s, gam, v1);
    iso_C(ew, lam, mu, s);
    symv(s, gam, v2);
  }
  const T k1 = lam + mu;
  const T k2 = mu * (gam[0] * gam[0] + gam[1] * gam[1] + gam[2] * gam[2]);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const T wg = k1 * (W[a][0] * gam[0] + W[a][1] * gam[1] + W[a][2] * gam[2]);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const T f = m[a] * v1[x] + P[a] * v2[x] + wg * gam[x] + k2 * W[a][x];
      qe[a][x] += f;
      en += ws[a][x] * f;
    }
  }
}

// One cut tet of Kuhn type t, one right-hand side: gathers, both sides, scatter-adds.
// t >= 0: compile-time Kuhn type; t < 0: the type trt given at run time
template <int t, bool TOTAL, bool SIG, typename T>
__device__ __forceinline__ void cut_tet(const typename Store<T>::type* __restrict__ dr,
                                        typename Store<T>::type* __restrict__ qr,
                                        const typename Store<T>::type* __restrict__ rec, const int4 nd,
                                        const int4 ej, long long N, int nX, const T (&ih)[3],
                                        const double* eps, T& en, T (&sg)[6], int trt = 0) {
  TetGrad<T> G;
  if constexpr (t < 0) {
    // g0 = -e_p/h_p, g1 = e_p/h_p - e_q/h_q, g2 = e_q/h_q - e_r/h_r, g3 = e_r/h_r, formed with
    // selects (no register array indexed at run time)
    const int p = perm_p(trt), q = perm_q(trt), r = perm_r(trt);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T ip = c == p ? ih[c] : T(0), iq = c == q ? ih[c] : T(0), ir = c == r ? ih[c] : T(0);
      G.g[0][c] = -ip;
      G.g[1][c] = ip - iq;
      G.g[2][c] = iq - ir;
      G.g[3][c] = ir;
    }
  }
  const int ndk[4] = {nd.x, nd.y, nd.z, nd.w};
  const int ejk[4] = {ej.x, ej.y, ej.z, ej.w};
  T ws[4][3];
  T es[6], ew[6];
  {
    T isd[12];
    ld_rec<3, T>(rec, isd);
    T us[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        us[a][c] = from_store<T>(dr[c * N + ndk[a]]);
        ws[a][c] = from_store<T>(dr[3 * N + (long long)c * nX + ejk[a]]) * isd[3 * a + c];
      }
    strain_of<t>(us, ih, G, es);
    strain_of<t>(ws, ih, G, ew);
  }
  // ed: the strain of d alone (the energy term); es also carries eps_bar in TOTAL mode
  T ed[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) ed[k] = es[k];
  if (TOTAL) {
    T E[6];
    mandel_to_tensor(eps, E);
#pragma unroll
    for (int k = 0; k < 6; ++k) es[k] += E[k];
  }
  T qs[4][3], qe[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) qs[a][c] = qe[a][c] = T(0);
  // the sides run one after the other except in FP64 (register pressure)
  constexpr int kSides = std::is_same<T, double>::value ? 2 : 1;
#pragma unroll kSides
  for (int si = 0; si < 2; ++si)
    cut_side<t, SIG>(rec + kRecSide + kRecSideLen * si, ws, es, ed, ew, ih, G, qs, qe, en, sg);
  T isd[12];
  ld_rec<3, T>(rec, isd);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(&qr[c * N + ndk[a]], to_store(qs[a][c]));
      atomicAdd(&qr[3 * N + (long long)c * nX + ejk[a]], to_store(qe[a][c] * isd[3 * a + c]));
    }
}

template <typename T>
__device__ __forceinline__ const typename Store<T>::type* cut_records(const CutData& cd);
template <>
__device__ __forceinline__ const float* cut_records<float>(const CutData& cd) {
  return cd.r32;
}
template <>
__device__ __forceinline__ const double* cut_records<double>(const CutData& cd) {
  return cd.r64;
}
template <>
__device__ __forceinline__ const double* cut_records<dw>(const CutData& cd) {
  return cd.r64;
}

// One thread per cut tet; the right-hand sides r0 .. r0+nr-1 are processed one after another
// inside the thread.  The block's 128 records are copied into shared memory with coalesced
// 16-byte loads (read from HBM once per launch) and read from there for every right-hand side.
// Per-RHS sums are reduced per warp each tet and kept in shared memory.
template <typename T, bool TOTAL, bool SIG>
__global__ void __launch_bounds__(kCutThreads, std::is_same<T, dw>::value ? 1
                                               : sizeof(T) == 8       ? 2
                                                                      : XFFT_CUT_MINB)
    k_apply_cut(const typename Store<T>::type* __restrict__ d, typename Store<T>::type* __restrict__ q,
                const CutData cd, const ApplyArgs a, int r0, int nr) {
  typedef typename Store<T>::type S;
  constexpr int NW = kCutThreads / 32;
  constexpr int RS = RecStride<S>::v;
  constexpr int kChunks = kRec * (int)sizeof(S) / 16;  // 16-byte pieces of a record
  __shared__ double acc[kCutMaxR][7][NW];
  extern __shared__ __align__(16) unsigned char cut_smem[];
  S* srec = reinterpret_cast<S*>(cut_smem);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kCutMaxR * 7 * NW; i += kCutThreads) (&acc[0][0][0])[i] = 0.0;
  if (a.units_cut && threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long n = 0;
    for (int rr = 0; rr < nr; ++rr) n += (!a.active || a.active[r0 + rr]) ? 1 : 0;
    atomicAdd(a.units_cut, n);
  }
  __syncthreads();
  const long long N = a.g.N;
  const int nX = a.nX;
  const int ncut = cd.ncut;
  const S* recs = cut_records<T>(cd);
  T ih[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ih[k] = (T)(1.0 / a.g.h[k]);
  for (int base = blockIdx.x * kCutThreads; base < ncut; base += gridDim.x * kCutThreads) {
    const int e = base + threadIdx.x;
    const bool ok = e < ncut;
    int t = 0;
    int4 nd = make_int4(0, 0, 0, 0), ej = nd;
    if (ok) {
      t = __ldg(cd.ip + 9 * ncut + e);
      nd = __ldg(cd.n4 + e);
      ej = __ldg(cd.e4 + e);
    }
    const S* rec;
    if (cut_staged<T>()) {
      const int nval = ncut - base < kCutThreads ? ncut - base : kCutThreads;
      const float4* src = reinterpret_cast<const float4*>(recs + (long long)base * kRec);
      __syncthreads();  // the previous group's records are no longer read
      for (int i = threadIdx.x; i < nval * kChunks; i += kCutThreads) {
        const int te = i / kChunks, ch = i - te * kChunks;
        *reinterpret_cast<float4*>(srec + te * RS + ch * (16 / (int)sizeof(S))) = __ldg(src + i);
      }
      __syncthreads();
      rec = srec + threadIdx.x * RS;
    } else {
      rec = recs + (long long)(ok ? e : 0) * kRec;
    }
    for (int rr = 0; rr < nr; ++rr) {
      const int rhs = r0 + rr;
      if (a.active && !a.active[rhs]) continue;  // uniform over the block
      T en = T(0);
      T sg[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
      if (ok) {
        const S* dr = d + rhs * a.stride;
        S* qr = q + rhs * a.stride;
        const double* eps = TOTAL ? a.eps + 6 * rhs : nullptr;
        if constexpr (std::is_same<T, dw>::value) {
          cut_tet<-1, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg, t);
        } else switch (t) {  // uniform over a warp except at the boundaries of the type groups
          case 0: cut_tet<0, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg); break;
          case 1: cut_tet<1, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg); break;
          case 2: cut_tet<2, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg); break;
          case 3: cut_tet<3, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg); break;
          case 4: cut_tet<4, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg); break;
          default: cut_tet<5, TOTAL, SIG, T>(dr, qr, rec, nd, ej, N, nX, ih, eps, en, sg); break;
        }
      }
      const double ew_sum = (double)warp_sum(red_val(en));
      if (lane == 0) acc[rr][0][wid] += ew_sum;
      if (SIG) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const double v = (double)warp_sum(red_val(sg[k]));
          if (lane == 0) acc[rr][1 + k][wid] += v;
        }
      }
    }
  }
  __syncthreads();
  const double r2 = 1.41421356237309504880;
  for (int i = threadIdx.x; i < nr * 7; i += kCutThreads) {
    const int rr = i / 7, k = i - rr * 7;
    const int rhs = r0 + rr;
    if (a.active && !a.active[rhs]) continue;
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += acc[rr][k][w];
    if (k >= 4) v *= r2;
    a.partials[((long long)rhs * 7 + k) * a.nparts + a.part_offset_cut + blockIdx.x] = v;
  }
}

}  // namespace xfft
