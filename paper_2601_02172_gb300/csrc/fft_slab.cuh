// Slab path of the FP32 X-FFT preconditioner (Sec. 4, eq. GreenHermitian) for square y-z planes
// of N x N nodes (N = 32, 48, 64, 80, 96, 128): three passes instead of five.
//
//   ks_fwd  one block per (rhs, component, x plane i): the n1 x n2 real plane (64 KB) is loaded
//           once (with the fused CG update f -= alpha q), transformed along z (real-to-complex by
//           row pairs) and along y entirely in shared memory, and stored as one packed plane.
//   kx_slab x transform, 3x3 Green solve with a precomputed factor table, inverse x transform,
//           on x lines gathered across the planes.
//   ks_inv  inverse y and z transforms of each plane, z = P^-1 f and the f^T z partial sums.
//
// Packed plane (n1/2 rows x n2 slots of complex values, the footprint of the real plane):
//   0 < k2 < n2/2: frequency (ky, k2) at row ky/2, slot k2 (ky even) or n2 - k2 (ky odd);
//   k2 = 0 and k2 = n2/2 (real z lines): the y transforms A (k2 = 0) and B (k2 = n2/2) of the
//   packed sequence F_j[0] + i F_j[n2/2]; position m of that line is row m/2, slot 0 (m even) or
//   n2/2 (m odd) and holds (A_0, B_0) at m = 0, (A_h, B_h) at m = h = n1/2, A_m for 0 < m < h and
//   B_{n1-m} for h < m < n1 (A and B are Hermitian in ky; the other halves are implied).
// The x lines are indexed by (row R, slot s); the packed real pairs at m = 0 and m = h (slot 0 of
// rows 0 and n1/4) are split into their two Hermitian spectra around the Green solve.
#pragma once

#include <cuda_runtime.h>

#include "fft_fast.cuh"
#include "xfft_kernels.h"

namespace xfft {
namespace slab {

using fast::cmul;
using fast::line_fft_map;
using fast::MapLoad;

// plane geometry for square y-z planes of n1 = n2 = N nodes (N divisible by 8, a planned length)
template <int N>
struct Sq {
  static constexpr int N1 = N;                      // y length
  static constexpr int N2 = N;                      // z length
  static constexpr int H2 = N2 / 2;
  static constexpr int PL = N1 * N2 / 2;            // complex values per packed plane
  static constexpr int RS = N2 + 1;                 // shared-memory row stride (odd: lines at distinct banks)
  static constexpr int E = N == 128 ? 16 : fast::Plan<N>::E;  // elements per thread of the y and z lines
  static constexpr int NT = N1 * N2 / (2 * E);      // threads of the plane kernels (512 at N = 128)
  static constexpr int MINB = NT >= 512 ? 2 : (768 / NT > 1 ? 768 / NT : 1);
  static_assert(N % 8 == 0 && N1 == N2, "square planes, 8-slot x tiles");
};
constexpr int kGF = 9;                     // floats per Green factor: il00, il11, il22, l10, l20, l21
#ifndef XFFT_KXS_ST
#define XFFT_KXS_ST 8
#endif
#ifndef XFFT_KXS_RG
#define XFFT_KXS_RG 2
#endif
constexpr int RG = XFFT_KXS_RG;            // right-hand sides per x-pass block
// x pass: elements per thread and block size for x length N0
template <int N0>
struct XCfg {
  // elements per thread of an x line (a multiple of every radix of the length's plan), so that
  // the block stays within 1024 threads
  static constexpr int EX = N0 == 128 || N0 == 256 ? 16 : N0 == 384 ? 24 : fast::Plan<N0>::E;
  // slots per x-pass block (XFFT_KXS_ST complex values: 8 = one 64-byte segment per plane), fewer
  // where the block would exceed 1024 threads
  static constexpr int ST = 3 * RG * XFFT_KXS_ST * (N0 / EX) <= 1024 ? XFFT_KXS_ST : 8;
  static constexpr int THREADS = 3 * RG * ST * (N0 / EX);
  static constexpr int MINB = THREADS <= 384 ? 2 : 1;
};

struct ZLine {  // row pair p as a contiguous complex line
  float2* base;
  __device__ __forceinline__ float2* at(int m) const { return base + m; }
};
struct RealPair {  // first forward z stage: rows 2p and 2p+1 as real and imaginary parts
  const float* r0;
  const float* r1;
  __device__ __forceinline__ float2 get(int m) const { return make_float2(r0[m], r1[m]); }
};
template <int N>
struct YLine {  // y line: even positions in slot s0, odd positions in slot s1
  float2* buf;
  int s0, s1;
  __device__ __forceinline__ float2* at(int m) const { return buf + (m >> 1) * Sq<N>::RS + ((m & 1) ? s1 : s0); }
};
template <int N>
__device__ __forceinline__ YLine<N> yline(float2* buf, int L) {
  YLine<N> y;
  y.buf = buf;
  y.s0 = L == 0 ? 0 : L;
  y.s1 = L == 0 ? Sq<N>::H2 : Sq<N>::N2 - L;
  return y;
}

// ---------------------------------------------------------------- forward plane pass
template <int N>
__global__ void __launch_bounds__(Sq<N>::NT, Sq<N>::MINB) ks_fwd(float* __restrict__ f, float2* __restrict__ spec,
                                              long long stride, long long sstride, int n0,
                                              const int* __restrict__ active,
                                              const float2* __restrict__ tw1, const float2* __restrict__ tw2,
                                              unsigned long long* __restrict__ units,
                                              const float* __restrict__ q, const RhsState* __restrict__ st) {
  constexpr int N1 = Sq<N>::N1, N2 = Sq<N>::N2, H2 = Sq<N>::H2, PL = Sq<N>::PL, RS = Sq<N>::RS;
  constexpr int E = Sq<N>::E, NT = Sq<N>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tws1 = reinterpret_cast<float2*>(smraw);
  float2* tws2 = tws1 + N1;
  float2* buf = tws2 + N2;
  float* bf = reinterpret_cast<float*>(buf);
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  if (units && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(units, 1ULL);
  const int c = blockIdx.x / n0, i = blockIdx.x - c * n0;
  const long long N3 = (long long)n0 * N1 * N2;
  float* fp = f + rhs * stride + c * N3 + (long long)i * N1 * N2;
  const float* qp = q ? q + rhs * stride + c * N3 + (long long)i * N1 * N2 : nullptr;
  const float alpha = q ? (float)st[rhs].alpha : 0.0f;
  for (int k = threadIdx.x; k < N1; k += NT) tws1[k] = tw1[k];
  for (int k = threadIdx.x; k < N2; k += NT) tws2[k] = tw2[k];
  constexpr int PER = N1 * N2 / NT;
  {
    float fv[PER], qv[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      fv[e] = fp[threadIdx.x + e * NT];
      qv[e] = q ? qp[threadIdx.x + e * NT] : 0.0f;
    }
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * NT;
      float v = fv[e];
      if (q) {
        v -= alpha * qv[e];  // fused CG update f -= alpha A d
        fp[idx] = v;
      }
      // real row j goes to the first (j even) or second half of line j/2 (stride RS complex)
      const int j = idx / N2, k = idx - j * N2;
      bf[2 * (j >> 1) * RS + (j & 1) * N2 + k] = v;
    }
  }
  __syncthreads();
  {  // z: one complex line per row pair (threads line-minor: a warp spans 32 lines)
    const int p = threadIdx.x % (N1 / 2), t = threadIdx.x / (N1 / 2);
    const RealPair ld0{bf + 2 * p * RS, bf + 2 * p * RS + N2};
    const ZLine mp{buf + p * RS};
    line_fft_map<float2, N2, E, false>(ld0, mp, tws2, t, true);
  }
  // split each row pair into its two half spectra (in place) and move the real k2 = 0 and
  // k2 = n2/2 values into the packed y line
  for (int idx = threadIdx.x; idx < (N1 / 2) * H2; idx += NT) {
    const int p = idx / H2, k = idx - p * H2;
    float2* row = buf + p * RS;
    if (k == 0) {
      const float2 a = row[0], b = row[H2];
      row[0] = make_float2(a.x, b.x);
      row[H2] = make_float2(a.y, b.y);
    } else {
      const float2 zk = row[k], zn = row[N2 - k];
      row[k] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
      row[N2 - k] = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    }
  }
  __syncthreads();
  {  // y: one line per k2 (threads line-minor: a warp touches consecutive slots)
    const int L = threadIdx.x % H2, t = threadIdx.x / H2;
    const YLine<N> mp = yline<N>(buf, L);
    line_fft_map<float2, N1, E, false>(MapLoad<float2, YLine<N>>{mp}, mp, tws1, t, true);
  }
  {  // split the packed line into A (k2 = 0) and B (k2 = n2/2)
    const YLine<N> sp = yline<N>(buf, 0);
    for (int m = 1 + threadIdx.x; m < N1 / 2; m += NT) {
      float2* pa = sp.at(m);
      float2* pb = sp.at(N1 - m);
      const float2 y0 = *pa, y1 = *pb;
      *pa = make_float2(0.5f * (y0.x + y1.x), 0.5f * (y0.y - y1.y));
      *pb = make_float2(0.5f * (y0.y + y1.y), -0.5f * (y0.x - y1.x));
    }
  }
  __syncthreads();
  float2* out = spec + rhs * sstride + ((long long)c * n0 + i) * PL;
  for (int k = threadIdx.x; k < PL; k += NT) {
    const int row = k / N2, sl = k - row * N2;
    out[k] = buf[row * RS + sl];
  }
}

// ---------------------------------------------------------------- inverse plane pass
template <int N>
__global__ void __launch_bounds__(Sq<N>::NT, Sq<N>::MINB) ks_inv(const float2* __restrict__ spec, const float* __restrict__ f,
                                              float* __restrict__ z, long long stride, long long sstride,
                                              int n0, float scale, const int* __restrict__ active,
                                              const float2* __restrict__ tw1, const float2* __restrict__ tw2,
                                              double* __restrict__ partials, int nparts) {
  constexpr int N1 = Sq<N>::N1, N2 = Sq<N>::N2, H2 = Sq<N>::H2, PL = Sq<N>::PL, RS = Sq<N>::RS;
  constexpr int E = Sq<N>::E, NT = Sq<N>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  float2* tws1 = reinterpret_cast<float2*>(smraw);
  float2* tws2 = tws1 + N1;
  float2* buf = tws2 + N2;
  const float* bf = reinterpret_cast<const float*>(buf);
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int c = blockIdx.x / n0, i = blockIdx.x - c * n0;
  for (int k = threadIdx.x; k < N1; k += NT) tws1[k] = tw1[k];
  for (int k = threadIdx.x; k < N2; k += NT) tws2[k] = tw2[k];
  {
    const float2* in = spec + rhs * sstride + ((long long)c * n0 + i) * PL;
    constexpr int PER = PL / NT;
    float2 v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) v[e] = in[threadIdx.x + e * NT];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int k = threadIdx.x + e * NT;
      const int row = k / N2, sl = k - row * N2;
      buf[row * RS + sl] = v[e];
    }
  }
  __syncthreads();
  {  // rebuild the packed y line Y = A + i B (both Hermitian in ky)
    const YLine<N> sp = yline<N>(buf, 0);
    for (int m = 1 + threadIdx.x; m < N1 / 2; m += NT) {
      float2* pa = sp.at(m);
      float2* pb = sp.at(N1 - m);
      const float2 A = *pa, B = *pb;
      *pa = make_float2(A.x - B.y, A.y + B.x);
      *pb = make_float2(A.x + B.y, B.x - A.y);
    }
  }
  __syncthreads();
  {
    const int L = threadIdx.x % H2, t = threadIdx.x / H2;
    const YLine<N> mp = yline<N>(buf, L);
    line_fft_map<float2, N1, E, true>(MapLoad<float2, YLine<N>>{mp}, mp, tws1, t, true);
  }
  // undo the packing of the real z lines and rebuild Z_k = X_k + i Y_k of each row pair
  for (int idx = threadIdx.x; idx < (N1 / 2) * H2; idx += NT) {
    const int p = idx / H2, k = idx - p * H2;
    float2* row = buf + p * RS;
    if (k == 0) {
      const float2 a = row[0], b = row[H2];
      row[0] = make_float2(a.x, b.x);
      row[H2] = make_float2(a.y, b.y);
    } else {
      const float2 X = row[k], Y = row[N2 - k];
      row[k] = make_float2(X.x - Y.y, X.y + Y.x);
      row[N2 - k] = make_float2(X.x + Y.y, Y.x - X.y);
    }
  }
  __syncthreads();
  {
    const int p = threadIdx.x % (N1 / 2), t = threadIdx.x / (N1 / 2);
    const ZLine mp{buf + p * RS};
    line_fft_map<float2, N2, E, true>(MapLoad<float2, ZLine>{mp}, mp, tws2, t, true);
  }
  const long long N3 = (long long)n0 * N1 * N2;
  const float* fp = f + rhs * stride + c * N3 + (long long)i * N1 * N2;
  float* zp = z + rhs * stride + c * N3 + (long long)i * N1 * N2;
  constexpr int PER = N1 * N2 / NT;
  float acc = 0.0f;
  {
    float fv[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) fv[e] = fp[threadIdx.x + e * NT];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * NT;
      const int j = idx / N2, k = idx - j * N2;
      // row j is the real (j even) or imaginary (j odd) part of line j/2
      const float val = bf[2 * ((j >> 1) * RS + k) + (j & 1)] * scale;
      zp[idx] = val;
      acc += val * fv[e];
    }
  }
  double vv[1] = {(double)acc}, tot[1];
  block_sum<1>(vv, red, tot);
  if (threadIdx.x == 0) partials[(long long)rhs * nparts + blockIdx.x] = tot[0];
}

// ---------------------------------------------------------------- Green factor table
// Frequency of x line (R, s) of the packed plane: ky, k2, and whether it is a packed real pair
// (then k2 = 0 for the A part and n2/2 for the B part).
template <int N>
__device__ __forceinline__ void line_freq(int R, int s, int& ky, int& k2, bool& pair) {
  constexpr int N1 = Sq<N>::N1, N2 = Sq<N>::N2, H2 = Sq<N>::H2;
  pair = false;
  if (s == 0 || s == H2) {
    const int m = 2 * R + (s == H2 ? 1 : 0);
    if (m == 0 || m == N1 / 2) {
      pair = true;
      ky = m;
      k2 = 0;
    } else if (m < N1 / 2) {
      ky = m;
      k2 = 0;
    } else {
      ky = N1 - m;
      k2 = H2;
    }
  } else if (s < H2) {
    ky = 2 * R;
    k2 = s;
  } else {
    ky = 2 * R + 1;
    k2 = N2 - s;
  }
}

// table[f][R][s][kx]: the Cholesky factor of the symbol at (kx, line (R, s)) (k2 = 0 for the
// packed pairs); a zero factor where the symbol vanishes (xi = 0)
template <int N>
__global__ void k_green_table(float* __restrict__ table, int n0, const float2* __restrict__ ge0,
                              const float2* __restrict__ ge1, const float2* __restrict__ ge2,
                              const float2* __restrict__ gs0, const float2* __restrict__ gs1,
                              const float2* __restrict__ gs2, float ih0, float ih1, float ih2,
                              float halfvol) {
  constexpr int N2 = Sq<N>::N2, PL = Sq<N>::PL;
  const long long n = (long long)n0 * PL;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int rs = (int)(idx / n0);
    const int kx = (int)(idx - (long long)rs * n0);
    const int R = rs / N2, s = rs - R * N2;
    int ky, k2;
    bool pair;
    line_freq<N>(R, s, ky, k2, pair);
    fast::GreenFactor<float2, float> gf;
    if (!fast::green_factor<float2, float>(gf, ge0[kx], ge1[ky], ge2[k2], gs0[kx], gs1[ky], gs2[k2], ih0,
                                           ih1, ih2, halfvol)) {
      gf.il00 = gf.il11 = gf.il22 = 0.0f;
      gf.l10 = gf.l20 = gf.l21 = make_float2(0.0f, 0.0f);
    }
    const float v[kGF] = {gf.il00, gf.il11, gf.il22, gf.l10.x, gf.l10.y, gf.l20.x, gf.l20.y, gf.l21.x, gf.l21.y};
#pragma unroll
    for (int k = 0; k < kGF; ++k) table[(long long)k * n + idx] = v[k];
  }
}

__device__ __forceinline__ fast::GreenFactor<float2, float> load_factor(const float* __restrict__ table,
                                                                        long long n, long long idx) {
  fast::GreenFactor<float2, float> gf;
  gf.il00 = table[idx];
  gf.il11 = table[n + idx];
  gf.il22 = table[2 * n + idx];
  gf.l10 = make_float2(table[3 * n + idx], table[4 * n + idx]);
  gf.l20 = make_float2(table[5 * n + idx], table[6 * n + idx]);
  gf.l21 = make_float2(table[7 * n + idx], table[8 * n + idx]);
  return gf;
}

__device__ __forceinline__ void solve_or_zero(const fast::GreenFactor<float2, float>& gf, float2& a, float2& b,
                                              float2& c) {
  fast::green_solve<float2, float>(gf, a, b, c);
}

// ---------------------------------------------------------------- x pass + Green
// block: row R, slots s0 .. s0+ST-1, right-hand sides r0 .. r0+RG-1 (blockIdx.x = group fastest
// so that the groups of one tile read the factor table from L2); lines (r, c, slot) of length N0.
template <int N0, int N>
__global__ void __launch_bounds__(XCfg<N0>::THREADS, XCfg<N0>::MINB)
    kx_slab(float2* __restrict__ spec, long long sstride, int n_rhs, int ngroups,
            const int* __restrict__ active, const float2* __restrict__ tw0, const float* __restrict__ table,
            const float2* __restrict__ ge0, const float2* __restrict__ ge1, const float2* __restrict__ ge2,
            const float2* __restrict__ gs0, const float2* __restrict__ gs1, const float2* __restrict__ gs2,
            float ih0, float ih1, float ih2, float halfvol) {
  constexpr int EX = XCfg<N0>::EX;
  constexpr int TL = N0 / EX;
  constexpr int LS = N0 + 1;
  constexpr int ST = XCfg<N0>::ST;
  constexpr int LINES = 3 * RG * ST;
  constexpr int NTX = LINES * TL;
  constexpr int N2 = Sq<N>::N2, H2 = Sq<N>::H2, PL = Sq<N>::PL;
  constexpr int TPR = N2 / ST;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int live[RG];
  const int grp = blockIdx.x % ngroups;
  const int tile = blockIdx.x / ngroups;
  const int R = tile / TPR, s0 = (tile - R * TPR) * ST;
  const int r0 = grp * RG;
  const int nr = min(RG, n_rhs - r0);
  int any = 0;
  for (int r = 0; r < nr; ++r) any |= (!active || active[r0 + r]) ? 1 : 0;
  if (!any) return;  // uniform per block
  if (threadIdx.x < RG) live[threadIdx.x] = (threadIdx.x < nr && (!active || active[r0 + threadIdx.x])) ? 1 : 0;
  float2* tws = reinterpret_cast<float2*>(smraw);
  float2* buf = tws + N0;
  for (int k = threadIdx.x; k < N0; k += NTX) tws[k] = tw0[k];
  __syncthreads();
  // element (line = (r * 3 + c) * ST + sl, i) at spec[(r0 + r) sstride + (c N0 + i) PL + R N2 + s0 + sl]
  {
    float2 v[EX];
#pragma unroll
    for (int e = 0; e < EX; ++e) {
      const int idx = threadIdx.x + e * NTX;
      const int sl = idx % ST, i = (idx / ST) % N0, rc = idx / (ST * N0);
      const int r = rc / 3, c = rc - 3 * r;
      v[e] = make_float2(0.0f, 0.0f);
      if (live[r]) v[e] = spec[(r0 + r) * sstride + ((long long)c * N0 + i) * PL + R * N2 + s0 + sl];
    }
#pragma unroll
    for (int e = 0; e < EX; ++e) {
      const int idx = threadIdx.x + e * NTX;
      const int sl = idx % ST, i = (idx / ST) % N0, rc = idx / (ST * N0);
      buf[(rc * ST + sl) * LS + i] = v[e];
    }
  }
  __syncthreads();
  // threads line-minor (a warp spans consecutive lines; LS odd keeps them on distinct banks)
  const int line = threadIdx.x % LINES, t = threadIdx.x / LINES;
  {
    const ZLine mp{buf + line * LS};
    line_fft_map<float2, N0, EX, false>(MapLoad<float2, ZLine>{mp}, mp, tws, t, true);
  }
  const long long ntab = (long long)N0 * PL;
  for (int it = threadIdx.x; it < ST * N0; it += NTX) {
    const int sl = it / N0, kx = it - sl * N0;
    const int s = s0 + sl;
    int ky, k2;
    bool pair;
    line_freq<N>(R, s, ky, k2, pair);
    const long long tidx = (long long)(R * N2 + s) * N0 + kx;
    if (!pair) {
      const fast::GreenFactor<float2, float> gf = load_factor(table, ntab, tidx);
      for (int r = 0; r < RG; ++r) {
        if (!live[r]) continue;
        float2* b0 = buf + ((r * 3 + 0) * ST + sl) * LS + kx;
        float2* b1 = buf + ((r * 3 + 1) * ST + sl) * LS + kx;
        float2* b2 = buf + ((r * 3 + 2) * ST + sl) * LS + kx;
        float2 F0 = *b0, F1 = *b1, F2 = *b2;
        solve_or_zero(gf, F0, F1, F2);
        *b0 = F0;
        *b1 = F1;
        *b2 = F2;
      }
    } else if (kx <= N0 / 2) {
      // packed real pair: Z = A + i B with A (k2 = 0) and B (k2 = n2/2) Hermitian in kx
      const int kn = kx == 0 ? 0 : N0 - kx;
      const fast::GreenFactor<float2, float> ga = load_factor(table, ntab, tidx);
      fast::GreenFactor<float2, float> gb;
      if (!fast::green_factor<float2, float>(gb, ge0[kx], ge1[ky], ge2[H2], gs0[kx], gs1[ky], gs2[H2], ih0, ih1,
                                             ih2, halfvol)) {
        gb.il00 = gb.il11 = gb.il22 = 0.0f;
        gb.l10 = gb.l20 = gb.l21 = make_float2(0.0f, 0.0f);
      }
      for (int r = 0; r < RG; ++r) {
        if (!live[r]) continue;
        float2 A[3], B[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 zk = buf[((r * 3 + c) * ST + sl) * LS + kx];
          const float2 zn = buf[((r * 3 + c) * ST + sl) * LS + kn];
          A[c] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
          B[c] = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
        }
        solve_or_zero(ga, A[0], A[1], A[2]);
        solve_or_zero(gb, B[0], B[1], B[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          buf[((r * 3 + c) * ST + sl) * LS + kx] = make_float2(A[c].x - B[c].y, A[c].y + B[c].x);
          buf[((r * 3 + c) * ST + sl) * LS + kn] = make_float2(A[c].x + B[c].y, B[c].x - A[c].y);
        }
      }
    }
  }
  __syncthreads();
  {
    const ZLine mp{buf + line * LS};
    line_fft_map<float2, N0, EX, true>(MapLoad<float2, ZLine>{mp}, mp, tws, t, true);
  }
#pragma unroll
  for (int e = 0; e < EX; ++e) {
    const int idx = threadIdx.x + e * NTX;
    const int sl = idx % ST, i = (idx / ST) % N0, rc = idx / (ST * N0);
    const int r = rc / 3, c = rc - 3 * r;
    if (live[r]) spec[(r0 + r) * sstride + ((long long)c * N0 + i) * PL + R * N2 + s0 + sl] = buf[(rc * ST + sl) * LS + i];
  }
}


static inline cudaError_t slab_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N>
cudaError_t green_table_n(float* table, int n0, const void* const* ge, const void* const* gs, const double* ih,
                          double halfvol, cudaStream_t s) {
  const long long n = (long long)n0 * Sq<N>::PL;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_green_table<N><<<blocks, 256, 0, s>>>(table, n0, (const float2*)ge[0], (const float2*)ge[1],
                                          (const float2*)ge[2], (const float2*)gs[0], (const float2*)gs[1],
                                          (const float2*)gs[2], (float)ih[0], (float)ih[1], (float)ih[2],
                                          (float)halfvol);
  return cudaGetLastError();
}

template <int N>
cudaError_t precondition_n(int n0, float* f, float* z, void* spec, long long stride, long long sstride,
                           const int* active, const void* tw0, const void* tw1, const void* tw2, const float* table,
                           const void* const* ge, const void* const* gs, const double* ih, double halfvol,
                           unsigned long long* units, const float* q, const RhsState* st, double* partials,
                           int nparts, int n_rhs, cudaStream_t s) {
  typedef Sq<N> Q;
  const size_t smp = sizeof(float2) * (Q::N1 + Q::N2 + (size_t)(Q::N1 / 2) * Q::RS);
  cudaError_t e = slab_smem((const void*)ks_fwd<N>, smp);
  if (e == cudaSuccess) e = slab_smem((const void*)ks_inv<N>, smp);
  if (e != cudaSuccess) return e;
  ks_fwd<N><<<dim3(3 * n0, n_rhs), Q::NT, smp, s>>>(f, (float2*)spec, stride, sstride, n0, active,
                                                    (const float2*)tw1, (const float2*)tw2, units, q, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ngroups = (n_rhs + RG - 1) / RG;
  switch (n0) {
#define X(n)                                                                                          \
  case n: {                                                                                           \
    const size_t smx = sizeof(float2) * (n + (size_t)3 * RG * XCfg<n>::ST * (n + 1));                \
    e = slab_smem((const void*)kx_slab<n, N>, smx);                                                   \
    if (e != cudaSuccess) return e;                                                                   \
    kx_slab<n, N><<<(Q::N1 / 2) * (Q::N2 / XCfg<n>::ST) * ngroups, XCfg<n>::THREADS, smx, s>>>(       \
        (float2*)spec, sstride, n_rhs, ngroups, active, (const float2*)tw0, table, (const float2*)ge[0], \
        (const float2*)ge[1], (const float2*)ge[2], (const float2*)gs[0], (const float2*)gs[1],        \
        (const float2*)gs[2], (float)ih[0], (float)ih[1], (float)ih[2], (float)halfvol);              \
    break;                                                                                            \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ks_inv<N><<<dim3(3 * n0, n_rhs), Q::NT, smp, s>>>((const float2*)spec, f, z, stride, sstride, n0,
                                                    (float)(1.0 / ((double)n0 * Q::N1 * Q::N2)), active,
                                                    (const float2*)tw1, (const float2*)tw2, partials, nparts);
  return cudaGetLastError();
}

#define XFFT_SLAB_DECL(N)                                                                                    \
  extern template cudaError_t green_table_n<N>(float*, int, const void* const*, const void* const*,          \
                                               const double*, double, cudaStream_t);                          \
  extern template cudaError_t precondition_n<N>(int, float*, float*, void*, long long, long long, const int*, \
                                                const void*, const void*, const void*, const float*,          \
                                                const void* const*, const void* const*, const double*, double, \
                                                unsigned long long*, const float*, const RhsState*, double*,  \
                                                int, int, cudaStream_t);
#define XFFT_SLAB_INST(N)                                                                                    \
  template cudaError_t green_table_n<N>(float*, int, const void* const*, const void* const*, const double*,   \
                                        double, cudaStream_t);                                                \
  template cudaError_t precondition_n<N>(int, float*, float*, void*, long long, long long, const int*,        \
                                         const void*, const void*, const void*, const float*,                 \
                                         const void* const*, const void* const*, const double*, double,       \
                                         unsigned long long*, const float*, const RhsState*, double*, int,    \
                                         int, cudaStream_t);
// plane sizes of the slab path; the 128 x 128 planes are instantiated in fft_slab.cu, the others in
// fft_slab_sq.cu (two translation units that build in parallel)
#define XFFT_SLAB_SMALL(X) X(32) X(48) X(64) X(80) X(96)

}  // namespace slab
}  // namespace xfft
