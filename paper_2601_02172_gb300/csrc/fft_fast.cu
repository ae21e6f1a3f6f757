// Fast path of the X-FFT preconditioner for grid lengths with a compile-time line plan
// (fft_fast.cuh): the same five passes as the generic path in fft.cu (z real-to-complex, y,
// x + Green + x inverse, y inverse, z complex-to-real with the f^T z sums), each line
// transformed by register-resident radix stages.
#include <cuda_runtime.h>

#include "fft_fast.cuh"
#include "xfft_kernels.h"

namespace xfft {

template <typename T>
struct Cplx;
template <>
struct Cplx<double> {
  typedef double2 type;
};
template <>
struct Cplx<float> {
  typedef float2 type;
};

namespace fast {

template <typename C>
__device__ __forceinline__ void load_table(C* dst, const C* __restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// ---------------------------------------------------------------- z axis, real -> complex
// Spectrum layout of the fast path: [c][k2][j][i] (x fastest), so that x lines are contiguous.
// Block: component c, row j, rows i0 .. i0 + 2 LPB - 1 (LPB row pairs, TL = N/E threads each).
template <typename T, int N>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && N == 384) ? 2 : 1) kz_r2c(T* __restrict__ f, typename Cplx<T>::type* __restrict__ spec,
                                              long long stride, long long sstride, int n0, int n1,
                                              int itiles, const int* __restrict__ active,
                                              const typename Cplx<T>::type* __restrict__ tw,
                                              unsigned long long* __restrict__ units,
                                              const T* __restrict__ q, const RhsState* __restrict__ st) {
  typedef typename Cplx<T>::type C;
  constexpr int TL = N / Plan<N>::E;
  constexpr int LPB = 256 / TL;
  constexpr int LS = N + 1;
  constexpr int K2 = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  if (units && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(units, 1ULL);
  C* tws = reinterpret_cast<C*>(smraw);
  C* buf = tws + N;
  load_table(tws, tw, N);
  const int it = blockIdx.x % itiles;
  const int cj = blockIdx.x / itiles;  // c * n1 + j
  const int c = cj / n1, j = cj - c * n1;
  const int i0 = it * 2 * LPB;
  const int nrows = min(2 * LPB, n0 - i0);
  const long long N3 = (long long)n0 * n1 * N;
  T* fr = f + rhs * stride + c * N3;
  const T* qr = q ? q + rhs * stride + c * N3 : nullptr;
  const T alpha = q ? (T)st[rhs].alpha : T(0);
  constexpr int PER = 2 * LPB * N / 256;  // = 2 E elements per thread (blockDim is 256)
  T fv[PER], qv[PER];
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int idx = threadIdx.x + e * 256;
    const int rl = idx / N, k = idx - rl * N;
    const long long o = ((long long)(i0 + rl) * n1 + j) * N + k;
    fv[e] = rl < nrows ? fr[o] : T(0);
    qv[e] = (q && rl < nrows) ? qr[o] : T(0);
  }
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int idx = threadIdx.x + e * 256;
    const int rl = idx / N, k = idx - rl * N;
    T v = fv[e];
    if (q && rl < nrows) {
      v -= alpha * qv[e];  // fused CG update f -= alpha A d
      fr[((long long)(i0 + rl) * n1 + j) * N + k] = v;
    }
    T* dst = reinterpret_cast<T*>(&buf[(rl >> 1) * LS + k]);
    dst[rl & 1] = v;
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, false>(buf + line * LS, tws, t);
  C* sp = spec + rhs * sstride + (long long)c * K2 * n1 * n0 + (long long)j * n0 + i0;
  for (int idx = threadIdx.x; idx < 2 * LPB * K2; idx += blockDim.x) {
    const int k = idx / (2 * LPB), rl = idx - k * (2 * LPB);
    if (rl >= nrows) continue;
    const int p = rl >> 1;
    const C zk = buf[p * LS + k];
    const C zn = buf[p * LS + (k == 0 ? 0 : N - k)];
    C out;
    if ((rl & 1) == 0) {  // X = (Z_k + conj Z_{N-k}) / 2
      out.x = T(0.5) * (zk.x + zn.x);
      out.y = T(0.5) * (zk.y - zn.y);
    } else {  // Y = (Z_k - conj Z_{N-k}) / (2i)
      out.x = T(0.5) * (zk.y + zn.y);
      out.y = T(-0.5) * (zk.x - zn.x);
    }
    sp[(long long)k * n1 * n0 + rl] = out;
  }
}

// ---------------------------------------------------------------- y axis (complex)
// block: (c, k2) slab, ti consecutive i columns; each column is a line along j of length N = n1
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(256) ky(typename Cplx<T>::type* __restrict__ spec, long long sstride,
                                          int n0, int ti, int ntiles, const int* __restrict__ active,
                                          const typename Cplx<T>::type* __restrict__ tw) {
  typedef typename Cplx<T>::type C;
  constexpr int TL = N / Plan<N>::E;
  constexpr int LS = N + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  C* tws = reinterpret_cast<C*>(smraw);
  C* buf = tws + N;
  load_table(tws, tw, N);
  const long long slab = blockIdx.x / ntiles;  // c * K2 + k2
  const int tile = blockIdx.x - (int)slab * ntiles;
  const int ii0 = tile * ti;
  const int tie = min(ti, n0 - ii0);
  C* sp = spec + rhs * sstride + slab * N * n0 + ii0;
  constexpr int E = Plan<N>::E;  // N ti elements over ti TL threads
  C v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = threadIdx.x + e * blockDim.x;
    const int j = idx / ti, kk = idx - j * ti;
    v[e].x = T(0);
    v[e].y = T(0);
    if (kk < tie) v[e] = sp[(long long)j * n0 + kk];
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = threadIdx.x + e * blockDim.x;
    const int j = idx / ti, kk = idx - j * ti;
    buf[kk * LS + j] = v[e];
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, INV>(buf + line * LS, tws, t);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = threadIdx.x + e * blockDim.x;
    const int j = idx / ti, kk = idx - j * ti;
    if (kk < tie) sp[(long long)j * n0 + kk] = buf[kk * LS + j];
  }
}

// ---------------------------------------------------------------- x axis + Green + inverse
#ifndef XFFT_KX_MAXT
#define XFFT_KX_MAXT 576  // FP32 x/Green kernel: largest block
#endif
#ifndef XFFT_KX_MINB
#define XFFT_KX_MINB 2  // FP32 x/Green kernel: resident blocks per SM asked of the compiler
#endif
template <typename T, int N>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : XFFT_KX_MAXT, sizeof(T) == 8 ? 1 : XFFT_KX_MINB)
    kx_green(typename Cplx<T>::type* __restrict__ spec, long long sstride, int n1, int K2, int rg,
             int n_rhs, const int* __restrict__ active, const typename Cplx<T>::type* __restrict__ tw,
             const typename Cplx<T>::type* __restrict__ ge0, const typename Cplx<T>::type* __restrict__ ge1,
             const typename Cplx<T>::type* __restrict__ ge2, const typename Cplx<T>::type* __restrict__ gs0,
             const typename Cplx<T>::type* __restrict__ gs1, const typename Cplx<T>::type* __restrict__ gs2,
             T ih0, T ih1, T ih2, T halfvol) {
  typedef typename Cplx<T>::type C;
  constexpr int TL = N / Plan<N>::E;
  constexpr int LS = N + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int live[64];
  const int r0 = blockIdx.y * rg;
  const int nr = min(rg, n_rhs - r0);
  int any = 0;
  for (int r = 0; r < nr; ++r) any |= (!active || active[r0 + r]) ? 1 : 0;
  if (!any) return;  // uniform per block
  if (threadIdx.x < nr) live[threadIdx.x] = (!active || active[r0 + threadIdx.x]) ? 1 : 0;
  C* tws = reinterpret_cast<C*>(smraw);
  C* buf = tws + N;
  load_table(tws, tw, N);
  const int k2 = blockIdx.x / n1;
  const int j = blockIdx.x - k2 * n1;
  const long long cstride = (long long)K2 * n1 * N;
  const long long off = ((long long)k2 * n1 + j) * N;
  const int lines = 3 * rg;
  __syncthreads();
  constexpr int E = Plan<N>::E;  // lines N elements over lines TL threads
  {
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int idx = threadIdx.x + e * blockDim.x;
      const int li = idx / N, i = idx - li * N;
      const int r = li / 3, c = li - 3 * r;
      v[e].x = T(0);
      v[e].y = T(0);
      if (r < nr && live[r]) v[e] = spec[(r0 + r) * sstride + c * cstride + off + i];
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int idx = threadIdx.x + e * blockDim.x;
      const int li = idx / N, i = idx - li * N;
      buf[li * LS + i] = v[e];
    }
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, false>(buf + line * LS, tws, t);
  const C e1 = ge1[j], s1 = gs1[j], e2 = ge2[k2], s2 = gs2[k2];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    GreenFactor<C, T> gf;
    const bool ok = green_factor<C, T>(gf, ge0[i], e1, e2, gs0[i], s1, s2, ih0, ih1, ih2, halfvol);
    for (int r = 0; r < nr; ++r) {
      C* b0 = buf + (3 * r + 0) * LS + i;
      C* b1 = buf + (3 * r + 1) * LS + i;
      C* b2 = buf + (3 * r + 2) * LS + i;
      C F0 = *b0, F1 = *b1, F2 = *b2;
      if (ok) {
        green_solve<C, T>(gf, F0, F1, F2);
      } else {
        F0.x = F0.y = F1.x = F1.y = F2.x = F2.y = T(0);
      }
      *b0 = F0;
      *b1 = F1;
      *b2 = F2;
    }
  }
  __syncthreads();
  line_fft<C, N, true>(buf + line * LS, tws, t);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = threadIdx.x + e * blockDim.x;
    const int li = idx / N, i = idx - li * N;
    const int r = li / 3, c = li - 3 * r;
    if (r < nr && live[r]) spec[(r0 + r) * sstride + c * cstride + off + i] = buf[li * LS + i];
  }
}

// ---------------------------------------------------------------- z axis, complex -> real
template <typename T, int N>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && N == 384) ? 2 : 1) kz_c2r(const typename Cplx<T>::type* __restrict__ spec,
                                              const T* __restrict__ f, T* __restrict__ z, long long stride,
                                              long long sstride, int n0, int n1, int itiles, T scale,
                                              const int* __restrict__ active,
                                              const typename Cplx<T>::type* __restrict__ tw,
                                              double* __restrict__ partials, int nparts) {
  typedef typename Cplx<T>::type C;
  constexpr int TL = N / Plan<N>::E;
  constexpr int LPB = 256 / TL;
  constexpr int LS = N + 1;
  constexpr int K2 = N / 2 + 1;
  constexpr int half = N / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  C* tws = reinterpret_cast<C*>(smraw);
  C* buf = tws + N;
  load_table(tws, tw, N);
  const int it = blockIdx.x % itiles;
  const int cj = blockIdx.x / itiles;
  const int c = cj / n1, j = cj - c * n1;
  const int i0 = it * 2 * LPB;
  const int nrows = min(2 * LPB, n0 - i0);
  const C* sp = spec + rhs * sstride + (long long)c * K2 * n1 * n0 + (long long)j * n0 + i0;
  // gather the half spectra of the row pairs: X (row 2p), Y (row 2p+1) at k2 = kk
  {
    constexpr int PER = (2 * LPB * K2 + 255) / 256;
    C v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * 256;
      const int kk = idx / (2 * LPB), rl = idx - kk * (2 * LPB);
      v[e].x = v[e].y = T(0);
      if (kk < K2 && rl < nrows) v[e] = sp[(long long)kk * n1 * n0 + rl];
    }
    // stage the half spectra (row rl, frequency kk) in the shared buffer
    T* tmp = reinterpret_cast<T*>(buf);
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * 256;
      const int kk = idx / (2 * LPB), rl = idx - kk * (2 * LPB);
      if (kk < K2) {
        tmp[(rl * K2 + kk) * 2 + 0] = v[e].x;
        tmp[(rl * K2 + kk) * 2 + 1] = (kk == 0 || kk == half) ? T(0) : v[e].y;
      }
    }
  }
  __syncthreads();
  // build Z_k = X_k + i Y_k for k < N from the staged half spectra (in registers, then store)
  C zv[Plan<N>::E];  // LPB * N / 256 = E values per thread
  {
    const T* tmp = reinterpret_cast<const T*>(buf);
    int q = 0;
    for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x, ++q) {
      const int p = idx / N, k = idx - p * N;
      const int kk = k <= half ? k : N - k;
      C X, Y;
      X.x = tmp[((2 * p) * K2 + kk) * 2 + 0];
      X.y = tmp[((2 * p) * K2 + kk) * 2 + 1];
      Y.x = tmp[((2 * p + 1) * K2 + kk) * 2 + 0];
      Y.y = tmp[((2 * p + 1) * K2 + kk) * 2 + 1];
      if (k > half) {
        X.y = -X.y;
        Y.y = -Y.y;
      }
      C Zc;
      Zc.x = X.x - Y.y;
      Zc.y = X.y + Y.x;
      zv[q] = Zc;
    }
  }
  __syncthreads();
  {
    int q = 0;
    for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x, ++q) {
      const int p = idx / N, k = idx - p * N;
      buf[p * LS + k] = zv[q];
    }
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, true>(buf + line * LS, tws, t);
  const long long N3 = (long long)n0 * n1 * N;
  const T* fr = f + rhs * stride + c * N3;
  T* zr = z + rhs * stride + c * N3;
  T tacc = T(0);
  {
    constexpr int PER = 2 * LPB * N / 256;
    T fv[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * 256;
      const int rl = idx / N, k = idx - rl * N;
      fv[e] = rl < nrows ? fr[((long long)(i0 + rl) * n1 + j) * N + k] : T(0);
    }
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * 256;
      const int rl = idx / N, k = idx - rl * N;
      if (rl < nrows) {
        const C v = buf[(rl >> 1) * LS + k];
        const T val = ((rl & 1) ? v.y : v.x) * scale;
        zr[((long long)(i0 + rl) * n1 + j) * N + k] = val;
        tacc += val * fv[e];
      }
    }
  }
  double vv[1] = {(double)tacc}, tot[1];
  block_sum<1>(vv, red, tot);
  if (threadIdx.x == 0) partials[(long long)rhs * nparts + blockIdx.x] = tot[0];
}

}  // namespace fast

// ---------------------------------------------------------------- host side

bool fast_fft_supported(int n) {
  switch (n) {
#define X(n) case n:
    XFFT_FAST_SIZES(X)
#undef X
    return true;
    default:
      return false;
  }
}

static int plan_E(int n) {
  switch (n) {
#define X(n) \
  case n:    \
    return fast::Plan<n>::E;
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return 1;
  }
}

int fast_threads_per_line(int n) { return n / plan_E(n); }

// row pairs per block of the z passes
int fast_z_pairs(int n2) { return 256 / fast_threads_per_line(n2); }

template <typename T>
static cudaError_t set_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
cudaError_t fast_z_r2c(int n2, T* f, void* spec, long long stride, long long sstride, int n0, int n1,
                       const int* active, const void* tw, unsigned long long* units, int n_rhs,
                       cudaStream_t s, const T* q, const RhsState* st) {
  typedef typename Cplx<T>::type C;
  switch (n2) {
#define X(n)                                                                                  \
  case n: {                                                                                   \
    constexpr int LPB = 256 / (n / fast::Plan<n>::E);                                          \
    const size_t sm = sizeof(C) * (n + (size_t)LPB * (n + 1));                                 \
    cudaError_t e = set_smem<T>((const void*)fast::kz_r2c<T, n>, sm);                          \
    if (e != cudaSuccess) return e;                                                           \
    const int itiles = (n0 + 2 * LPB - 1) / (2 * LPB);                                         \
    fast::kz_r2c<T, n><<<dim3(3 * n1 * itiles, n_rhs), 256, sm, s>>>(                          \
        f, (C*)spec, stride, sstride, n0, n1, itiles, active, (const C*)tw, units, q, st);      \
    return cudaGetLastError();                                                                \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

// number of blocks of one z pass (and partial-sum slots of the complex-to-real pass)
int fast_z_blocks(int n0, int n1, int n2) {
  switch (n2) {
#define X(n)                                                          \
  case n: {                                                           \
    constexpr int LPB = 256 / (n / fast::Plan<n>::E);                  \
    return 3 * n1 * ((n0 + 2 * LPB - 1) / (2 * LPB));                  \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return 0;
  }
}

template <typename T>
cudaError_t fast_z_c2r(int n2, const void* spec, const T* f, T* z, long long stride, long long sstride,
                       int n0, int n1, double scale, const int* active, const void* tw, double* partials,
                       int nparts, int n_rhs, cudaStream_t s) {
  typedef typename Cplx<T>::type C;
  switch (n2) {
#define X(n)                                                                                  \
  case n: {                                                                                   \
    constexpr int LPB = 256 / (n / fast::Plan<n>::E);                                          \
    const size_t sm = sizeof(C) * (n + (size_t)LPB * (n + 2));                                 \
    cudaError_t e = set_smem<T>((const void*)fast::kz_c2r<T, n>, sm);                          \
    if (e != cudaSuccess) return e;                                                           \
    const int itiles = (n0 + 2 * LPB - 1) / (2 * LPB);                                         \
    fast::kz_c2r<T, n><<<dim3(3 * n1 * itiles, n_rhs), 256, sm, s>>>(                          \
        (const C*)spec, f, z, stride, sstride, n0, n1, itiles, (T)scale, active, (const C*)tw,  \
        partials, nparts);                                                                    \
    return cudaGetLastError();                                                                \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T, bool INV>
cudaError_t fast_y(int n1, int n0, void* spec, long long sstride, int K2, const int* active,
                   const void* tw, int n_rhs, cudaStream_t s) {
  typedef typename Cplx<T>::type C;
  switch (n1) {
#define X(n)                                                                                  \
  case n: {                                                                                   \
    constexpr int TL = n / fast::Plan<n>::E;                                                   \
    constexpr int TIMAX = 256 / TL;                                                            \
    const int ntiles = (n0 + TIMAX - 1) / TIMAX;                                               \
    const int ti = (n0 + ntiles - 1) / ntiles;                                                 \
    const size_t sm = sizeof(C) * (n + (size_t)ti * (n + 1));                                  \
    cudaError_t e = set_smem<T>((const void*)fast::ky<T, n, INV>, sm);                         \
    if (e != cudaSuccess) return e;                                                           \
    fast::ky<T, n, INV><<<dim3(3 * K2 * ntiles, n_rhs), ti * TL, sm, s>>>(                     \
        (C*)spec, sstride, n0, ti, ntiles, active, (const C*)tw);                              \
    return cudaGetLastError();                                                                \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t fast_x_green(int n0, int n1, void* spec, long long sstride, int K2, const int* active,
                         const void* tw, const void* const* ge, const void* const* gs, const double* ih,
                         double halfvol, int n_rhs, cudaStream_t s) {
  typedef typename Cplx<T>::type C;
  switch (n0) {
#define X(n)                                                                                    \
  case n: {                                                                                     \
    constexpr int TL = n / fast::Plan<n>::E;                                                     \
    const int maxthr = sizeof(T) == 8 ? 384 : XFFT_KX_MAXT;                                      \
    int lmax = maxthr / TL; /* lines per block */                                                \
    while (lmax > 3 && sizeof(C) * (n + (size_t)lmax * (n + 1)) > 160 * 1024) --lmax;            \
    int rg = n_rhs < lmax / 3 ? n_rhs : lmax / 3;                                                \
    if (rg < 1) rg = 1;                                                                          \
    const int ngroups = (n_rhs + rg - 1) / rg;                                                   \
    const size_t sm = sizeof(C) * (n + 3 * (size_t)rg * (n + 1));                                \
    cudaError_t e = set_smem<T>((const void*)fast::kx_green<T, n>, sm);                          \
    if (e != cudaSuccess) return e;                                                             \
    fast::kx_green<T, n><<<dim3(n1 * K2, ngroups), 3 * rg * TL, sm, s>>>(                        \
        (C*)spec, sstride, n1, K2, rg, n_rhs, active, (const C*)tw, (const C*)ge[0],             \
        (const C*)ge[1], (const C*)ge[2], (const C*)gs[0], (const C*)gs[1], (const C*)gs[2],      \
        (T)ih[0], (T)ih[1], (T)ih[2], (T)halfvol);                                               \
    return cudaGetLastError();                                                                  \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

#define XFFT_INST(T)                                                                                  \
  template cudaError_t fast_z_r2c<T>(int, T*, void*, long long, long long, int, int, const int*,       \
                                     const void*, unsigned long long*, int, cudaStream_t, const T*,   \
                                     const RhsState*);                                                \
  template cudaError_t fast_z_c2r<T>(int, const void*, const T*, T*, long long, long long, int, int,   \
                                     double, const int*, const void*, double*, int, int, cudaStream_t); \
  template cudaError_t fast_y<T, false>(int, int, void*, long long, int, const int*, const void*, int, \
                                        cudaStream_t);                                                \
  template cudaError_t fast_y<T, true>(int, int, void*, long long, int, const int*, const void*, int,  \
                                       cudaStream_t);                                                 \
  template cudaError_t fast_x_green<T>(int, int, void*, long long, int, const int*, const void*,      \
                                       const void* const*, const void* const*, const double*, double, \
                                       int, cudaStream_t);
XFFT_INST(float)
XFFT_INST(double)
#undef XFFT_INST

}  // namespace xfft
