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
// block: LPB row pairs, TL = N/E threads per pair
template <typename T, int N>
__global__ void __launch_bounds__(256) kz_r2c(const T* __restrict__ f, typename Cplx<T>::type* __restrict__ spec,
                                              long long stride, long long sstride, long long rows,
                                              const int* __restrict__ active,
                                              const typename Cplx<T>::type* __restrict__ tw,
                                              unsigned long long* __restrict__ units) {
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
  const long long row0 = 2LL * blockIdx.x * LPB;
  const int nrows = (int)min((long long)2 * LPB, rows - row0);
  const T* fr = f + rhs * stride + row0 * N;
  for (int idx = threadIdx.x; idx < 2 * LPB * N; idx += blockDim.x) {
    const int rl = idx / N, k = idx - rl * N;
    const T v = rl < nrows ? fr[(long long)rl * N + k] : T(0);
    T* dst = reinterpret_cast<T*>(&buf[(rl >> 1) * LS + k]);
    dst[rl & 1] = v;
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, false>(buf + line * LS, tws, t);
  C* sp = spec + rhs * sstride + row0 * K2;
  for (int idx = threadIdx.x; idx < LPB * K2; idx += blockDim.x) {
    const int p = idx / K2, k = idx - p * K2;
    if (2 * p >= nrows) continue;
    const C zk = buf[p * LS + k];
    const C zn = buf[p * LS + (k == 0 ? 0 : N - k)];
    C X, Y;
    X.x = T(0.5) * (zk.x + zn.x);
    X.y = T(0.5) * (zk.y - zn.y);
    Y.x = T(0.5) * (zk.y + zn.y);
    Y.y = T(-0.5) * (zk.x - zn.x);
    sp[(long long)(2 * p) * K2 + k] = X;
    if (2 * p + 1 < nrows) sp[(long long)(2 * p + 1) * K2 + k] = Y;
  }
}

// ---------------------------------------------------------------- y axis (complex)
// block: TK lines (consecutive k2 of one (c, i) slab), TL threads per line
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(256) ky(typename Cplx<T>::type* __restrict__ spec, long long sstride,
                                          int K2, int tk, int ntiles, const int* __restrict__ active,
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
  const long long slab = blockIdx.x / ntiles;
  const int tile = blockIdx.x - (int)slab * ntiles;
  const int k0 = tile * tk;
  const int tke = min(tk, K2 - k0);
  C* sp = spec + rhs * sstride + slab * N * K2 + k0;
  for (int idx = threadIdx.x; idx < N * tk; idx += blockDim.x) {
    const int j = idx / tk, kk = idx - j * tk;
    C v;
    v.x = T(0);
    v.y = T(0);
    if (kk < tke) v = sp[(long long)j * K2 + kk];
    buf[kk * LS + j] = v;
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, INV>(buf + line * LS, tws, t);
  for (int idx = threadIdx.x; idx < N * tk; idx += blockDim.x) {
    const int j = idx / tk, kk = idx - j * tk;
    if (kk < tke) sp[(long long)j * K2 + kk] = buf[kk * LS + j];
  }
}

// ---------------------------------------------------------------- x axis + Green + inverse
template <typename C, typename T>
__device__ __forceinline__ void green3(C& F0, C& F1, C& F2, C e0, C e1, C e2, C s0, C s1, C s2, T ih0,
                                       T ih1, T ih2, T halfvol) {
  C g[3];
  g[0].x = s0.x * ih0;
  g[0].y = s0.y * ih0;
  g[1].x = s1.x * ih1;
  g[1].y = s1.y * ih1;
  g[2].x = s2.x * ih2;
  g[2].y = s2.y * ih2;
  const T a0 = g[0].x * g[0].x + g[0].y * g[0].y;
  const T a1 = g[1].x * g[1].x + g[1].y * g[1].y;
  const T a2 = g[2].x * g[2].x + g[2].y * g[2].y;
  const T S = a0 + a1 + a2;
  C zero;
  zero.x = T(0);
  zero.y = T(0);
  if (!(S > T(0))) {
    F0 = F1 = F2 = zero;
    return;
  }
  const C e[3] = {e0, e1, e2};
  C m01 = zero, m02 = zero, m12 = zero;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int p = perm_p(t), q = perm_q(t), r = perm_r(t);
    C G[3];
    G[p] = g[p];
    G[q] = cmul(e[p], g[q]);
    G[r] = cmul(cmul(e[p], e[q]), g[r]);
    m01 = cadd(m01, cmulc(G[0], G[1]));
    m02 = cadd(m02, cmulc(G[0], G[2]));
    m12 = cadd(m12, cmulc(G[1], G[2]));
  }
  const T d0 = halfvol * T(6) * (S + a0);
  const T d1 = halfvol * T(6) * (S + a1);
  const T d2 = halfvol * T(6) * (S + a2);
  m01.x *= halfvol;
  m01.y *= halfvol;
  m02.x *= halfvol;
  m02.y *= halfvol;
  m12.x *= halfvol;
  m12.y *= halfvol;
  // Cholesky M = L L^H with M(1,0) = conj(m01), M(2,0) = conj(m02), M(2,1) = conj(m12)
  const T il00 = T(1) / sqrt(d0);
  C l10, l20, l21;
  l10.x = m01.x * il00;
  l10.y = -m01.y * il00;
  l20.x = m02.x * il00;
  l20.y = -m02.y * il00;
  const T l11sq = d1 - (l10.x * l10.x + l10.y * l10.y);
  if (!(l11sq > T(0))) {
    F0 = F1 = F2 = zero;
    return;
  }
  const T il11 = T(1) / sqrt(l11sq);
  C m21;
  m21.x = m12.x;
  m21.y = -m12.y;
  const C t21 = csub(m21, cmulc(l20, l10));
  l21.x = t21.x * il11;
  l21.y = t21.y * il11;
  const T l22sq = d2 - (l20.x * l20.x + l20.y * l20.y) - (l21.x * l21.x + l21.y * l21.y);
  if (!(l22sq > T(0))) {
    F0 = F1 = F2 = zero;
    return;
  }
  const T il22 = T(1) / sqrt(l22sq);
  C y0, y1, y2, t;
  y0.x = F0.x * il00;
  y0.y = F0.y * il00;
  t = csub(F1, cmul(l10, y0));
  y1.x = t.x * il11;
  y1.y = t.y * il11;
  t = csub(csub(F2, cmul(l20, y0)), cmul(l21, y1));
  y2.x = t.x * il22;
  y2.y = t.y * il22;
  C x0, x1, x2;
  x2.x = y2.x * il22;
  x2.y = y2.y * il22;
  t = csub(y1, cmulc(x2, l21));
  x1.x = t.x * il11;
  x1.y = t.y * il11;
  t = csub(csub(y0, cmulc(x1, l10)), cmulc(x2, l20));
  x0.x = t.x * il00;
  x0.y = t.y * il00;
  F0 = x0;
  F1 = x1;
  F2 = x2;
}

// block: j, a k2 tile of width tk, all three components: 3 tk lines of length N = n0
template <typename T, int N>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : 768) kx_green(typename Cplx<T>::type* __restrict__ spec, long long sstride,
                                                 int n1, int K2, int tk, int ntiles,
                                                 const int* __restrict__ active,
                                                 const typename Cplx<T>::type* __restrict__ tw,
                                                 const typename Cplx<T>::type* __restrict__ ge0,
                                                 const typename Cplx<T>::type* __restrict__ ge1,
                                                 const typename Cplx<T>::type* __restrict__ ge2,
                                                 const typename Cplx<T>::type* __restrict__ gs0,
                                                 const typename Cplx<T>::type* __restrict__ gs1,
                                                 const typename Cplx<T>::type* __restrict__ gs2, T ih0,
                                                 T ih1, T ih2, T halfvol) {
  typedef typename Cplx<T>::type C;
  constexpr int TL = N / Plan<N>::E;
  constexpr int LS = N + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  C* tws = reinterpret_cast<C*>(smraw);
  C* buf = tws + N;
  load_table(tws, tw, N);
  const int j = blockIdx.x / ntiles;
  const int tile = blockIdx.x - j * ntiles;
  const int k0 = tile * tk;
  const int tke = min(tk, K2 - k0);
  C* sp = spec + rhs * sstride;
  const long long cstride = (long long)N * n1 * K2;
  const long long istride = (long long)n1 * K2;
  for (int idx = threadIdx.x; idx < 3 * N * tk; idx += blockDim.x) {
    const int ci = idx / tk, kk = idx - ci * tk;
    const int c = ci / N, i = ci - c * N;
    C v;
    v.x = T(0);
    v.y = T(0);
    if (kk < tke) v = sp[c * cstride + i * istride + (long long)j * K2 + k0 + kk];
    buf[(c * tk + kk) * LS + i] = v;
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, false>(buf + line * LS, tws, t);
  const C e1 = ge1[j], s1 = gs1[j];
  for (int idx = threadIdx.x; idx < N * tk; idx += blockDim.x) {
    const int kk = idx / N, i = idx - kk * N;
    if (kk >= tke) continue;
    C F0 = buf[(0 * tk + kk) * LS + i];
    C F1 = buf[(1 * tk + kk) * LS + i];
    C F2 = buf[(2 * tk + kk) * LS + i];
    green3<C, T>(F0, F1, F2, ge0[i], e1, ge2[k0 + kk], gs0[i], s1, gs2[k0 + kk], ih0, ih1, ih2, halfvol);
    buf[(0 * tk + kk) * LS + i] = F0;
    buf[(1 * tk + kk) * LS + i] = F1;
    buf[(2 * tk + kk) * LS + i] = F2;
  }
  __syncthreads();
  line_fft<C, N, true>(buf + line * LS, tws, t);
  for (int idx = threadIdx.x; idx < 3 * N * tk; idx += blockDim.x) {
    const int ci = idx / tk, kk = idx - ci * tk;
    const int c = ci / N, i = ci - c * N;
    if (kk < tke) sp[c * cstride + i * istride + (long long)j * K2 + k0 + kk] = buf[(c * tk + kk) * LS + i];
  }
}

// ---------------------------------------------------------------- z axis, complex -> real
template <typename T, int N>
__global__ void __launch_bounds__(256) kz_c2r(const typename Cplx<T>::type* __restrict__ spec,
                                              const T* __restrict__ f, T* __restrict__ z, long long stride,
                                              long long sstride, long long rows, T scale,
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
  const long long row0 = 2LL * blockIdx.x * LPB;
  const int nrows = (int)min((long long)2 * LPB, rows - row0);
  const C* sp = spec + rhs * sstride + row0 * K2;
  for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
    const int p = idx / N, k = idx - p * N;
    C X, Y;
    X.x = X.y = Y.x = Y.y = T(0);
    if (2 * p < nrows) {
      const int kk = k <= half ? k : N - k;
      X = sp[(long long)(2 * p) * K2 + kk];
      if (2 * p + 1 < nrows) Y = sp[(long long)(2 * p + 1) * K2 + kk];
      if (k == 0 || k == half) {
        X.y = T(0);
        Y.y = T(0);
      } else if (k > half) {
        X.y = -X.y;
        Y.y = -Y.y;
      }
    }
    C Zc;
    Zc.x = X.x - Y.y;
    Zc.y = X.y + Y.x;
    buf[p * LS + k] = Zc;
  }
  __syncthreads();
  const int line = threadIdx.x / TL, t = threadIdx.x - line * TL;
  line_fft<C, N, true>(buf + line * LS, tws, t);
  const T* fr = f + rhs * stride + row0 * N;
  T* zr = z + rhs * stride + row0 * N;
  T tacc = T(0);
  for (int idx = threadIdx.x; idx < nrows * N; idx += blockDim.x) {
    const int rl = idx / N, k = idx - rl * N;
    const C v = buf[(rl >> 1) * LS + k];
    const T val = ((rl & 1) ? v.y : v.x) * scale;
    zr[(long long)rl * N + k] = val;
    tacc += val * fr[(long long)rl * N + k];
  }
  double vv[1] = {(double)tacc}, tot[1];
  block_sum<1>(vv, red, tot);
  if (threadIdx.x == 0) partials[(long long)rhs * nparts + blockIdx.x] = tot[0];
}

}  // namespace fast

// ---------------------------------------------------------------- host side
#define XFFT_FAST_SIZES(X) X(16) X(32) X(48) X(64) X(80) X(96) X(128) X(192) X(256) X(384)

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
cudaError_t fast_z_r2c(int n2, const T* f, void* spec, long long stride, long long sstride, long long rows,
                       const int* active, const void* tw, unsigned long long* units, int n_rhs,
                       cudaStream_t s) {
  typedef typename Cplx<T>::type C;
  switch (n2) {
#define X(n)                                                                                  \
  case n: {                                                                                   \
    constexpr int LPB = 256 / (n / fast::Plan<n>::E);                                          \
    const size_t sm = sizeof(C) * (n + (size_t)LPB * (n + 1));                                 \
    cudaError_t e = set_smem<T>((const void*)fast::kz_r2c<T, n>, sm);                          \
    if (e != cudaSuccess) return e;                                                           \
    const long long nb = (rows + 2 * LPB - 1) / (2 * LPB);                                     \
    fast::kz_r2c<T, n><<<dim3((unsigned)nb, n_rhs), 256, sm, s>>>(                             \
        f, (C*)spec, stride, sstride, rows, active, (const C*)tw, units);                      \
    return cudaGetLastError();                                                                \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t fast_z_c2r(int n2, const void* spec, const T* f, T* z, long long stride, long long sstride,
                       long long rows, double scale, const int* active, const void* tw,
                       double* partials, int nparts, int n_rhs, cudaStream_t s) {
  typedef typename Cplx<T>::type C;
  switch (n2) {
#define X(n)                                                                                  \
  case n: {                                                                                   \
    constexpr int LPB = 256 / (n / fast::Plan<n>::E);                                          \
    const size_t sm = sizeof(C) * (n + (size_t)LPB * (n + 1));                                 \
    cudaError_t e = set_smem<T>((const void*)fast::kz_c2r<T, n>, sm);                          \
    if (e != cudaSuccess) return e;                                                           \
    const long long nb = (rows + 2 * LPB - 1) / (2 * LPB);                                     \
    fast::kz_c2r<T, n><<<dim3((unsigned)nb, n_rhs), 256, sm, s>>>(                             \
        (const C*)spec, f, z, stride, sstride, rows, (T)scale, active, (const C*)tw, partials,  \
        nparts);                                                                              \
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
    constexpr int TKMAX = 256 / TL;                                                            \
    const int ntiles = (K2 + TKMAX - 1) / TKMAX;                                               \
    const int tk = (K2 + ntiles - 1) / ntiles;                                                 \
    const size_t sm = sizeof(C) * (n + (size_t)tk * (n + 1));                                  \
    cudaError_t e = set_smem<T>((const void*)fast::ky<T, n, INV>, sm);                         \
    if (e != cudaSuccess) return e;                                                           \
    fast::ky<T, n, INV><<<dim3(3 * n0 * ntiles, n_rhs), tk * TL, sm, s>>>(                     \
        (C*)spec, sstride, K2, tk, ntiles, active, (const C*)tw);                              \
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
#define X(n)                                                                                  \
  case n: {                                                                                   \
    constexpr int TL = n / fast::Plan<n>::E;                                                   \
    int tkmax = (sizeof(T) == 8 ? 384 : 768) / (3 * TL);                                       \
    if (tkmax > 16) tkmax = 16;                                                                \
    while (tkmax > 1 && sizeof(C) * (n + 3 * (size_t)tkmax * (n + 1)) > 160 * 1024) --tkmax;    \
    const int ntiles = (K2 + tkmax - 1) / tkmax;                                               \
    const int tk = (K2 + ntiles - 1) / ntiles;                                                 \
    const size_t sm = sizeof(C) * (n + 3 * (size_t)tk * (n + 1));                              \
    cudaError_t e = set_smem<T>((const void*)fast::kx_green<T, n>, sm);                        \
    if (e != cudaSuccess) return e;                                                           \
    fast::kx_green<T, n><<<dim3(n1 * ntiles, n_rhs), 3 * tk * TL, sm, s>>>(                    \
        (C*)spec, sstride, n1, K2, tk, ntiles, active, (const C*)tw, (const C*)ge[0],          \
        (const C*)ge[1], (const C*)ge[2], (const C*)gs[0], (const C*)gs[1], (const C*)gs[2],    \
        (T)ih[0], (T)ih[1], (T)ih[2], (T)halfvol);                                             \
    return cudaGetLastError();                                                                \
  }
    XFFT_FAST_SIZES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

#define XFFT_INST(T)                                                                                  \
  template cudaError_t fast_z_r2c<T>(int, const T*, void*, long long, long long, long long, const int*, \
                                     const void*, unsigned long long*, int, cudaStream_t);            \
  template cudaError_t fast_z_c2r<T>(int, const void*, const T*, T*, long long, long long, long long,  \
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
