// X-FFT preconditioner P^{-1} = diag(A0_11^{-1}, I) (eqs. scaledPreconditioner,
// constantCoefficientPreconditioner, GreenHermitian).
//
// The constant-coefficient operator A0_11 = int grad^s N_FE : grad^s N_FE is a periodic
// convolution, diagonalised by the 3D DFT into 3x3 Hermitian blocks
//   M(xi) = Z(xi)^H A0_11,v Z(xi),   Z = c(xi) (x) I_3,   c_j = exp(i theta . Y_j),
// theta_a = 2 pi xi_a / n_a.  Summing the six Kuhn tets in closed form gives
//   M(xi) = (|T| / 2) sum_tets ( |G|^2 I + G G^H ),   G = sum_a c_a grad N_a,
// and for the tet (p,q,r): G_p = s_p/h_p, G_q = e_p s_q/h_q, G_r = e_p e_q s_r/h_r with
// e_a = exp(i theta_a), s_a = e_a - 1.  The inverse is applied per frequency by a 3x3 complex
// Cholesky solve; xi = 0 maps to 0 (mean-free standard part).
//
// The 3D transform is hand written: a mixed-radix (4, 2, 3, 5) Stockham FFT in shared memory.
//   pass 1  z axis, real-to-complex (two real rows packed as one complex row)
//   pass 2  y axis, complex
//   pass 3  x axis forward, Green solve of the three components, x axis inverse
//   pass 4  y axis inverse
//   pass 5  z axis complex-to-real, scaled by 1/N, fused f^T z partial sums
// The enriched block of P is the identity (scaled enriched DOFs), applied with its f^T f sum.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "xfft_kernels.h"

namespace xfft {

constexpr int kMaxStages = 14;

struct AxisPlan {
  int n;
  int nst;
  int rad[kMaxStages];
};

struct FftPlan {
  GridDev g;
  int n[3];
  int K2;
  AxisPlan ax[3];
  double2* twd[3];
  float2* twf[3];
  double2* ged[3];  // e_a(xi)
  double2* gsd[3];  // e_a(xi) - 1
  float2* gef[3];
  float2* gsf[3];
  int xpairs;       // row pairs per block in the z passes
  int ytk_d, ytiles_d, ytk_f, ytiles_f;  // k2 tile in the y passes (double / float)
  int gtk_d, gtiles_d, gtk_f, gtiles_f;  // k2 tile in the Green pass (double / float)
  bool fast;        // every axis has a compile-time line plan (fft_fast.cu)
  bool slab;        // FP32 y-z plane path (fft_slab.cu)
  float* gtab;      // its Green factor table
  void* pool;
};

// slab path (fft_slab.cu)
bool slab_supported(int n0, int n1, int n2);
size_t slab_table_floats(int n0, int n1);
int slab_z_blocks(int n0);
cudaError_t slab_green_table(float* table, int n0, int n1, const void* const* ge, const void* const* gs,
                             const double* ih, double halfvol, cudaStream_t s);
cudaError_t slab_precondition(int n0, int n1, float* f, float* z, void* spec, long long stride, long long sstride,
                              const int* active, const void* tw0, const void* tw1, const void* tw2,
                              const float* table, const void* const* ge, const void* const* gs,
                              const double* ih, double halfvol, unsigned long long* units, const float* q,
                              const RhsState* st, double* partials, int nparts, int n_rhs, cudaStream_t s);

// fast path (fft_fast.cu)
bool fast_fft_supported(int n);
int fast_z_pairs(int n2);
template <typename T>
cudaError_t fast_z_r2c(int n2, T* f, void* spec, long long stride, long long sstride, int n0, int n1,
                       const int* active, const void* tw, unsigned long long* units, int n_rhs,
                       cudaStream_t s, const T* q, const RhsState* st);
template <typename T>
cudaError_t fast_z_c2r(int n2, const void* spec, const T* f, T* z, long long stride, long long sstride,
                       int n0, int n1, double scale, const int* active, const void* tw,
                       double* partials, int nparts, int n_rhs, cudaStream_t s);
int fast_z_blocks(int n0, int n1, int n2);
template <typename T, bool INV>
cudaError_t fast_y(int n1, int n0, void* spec, long long sstride, int K2, const int* active,
                   const void* tw, int n_rhs, cudaStream_t s);
template <typename T>
cudaError_t fast_x_green(int n0, int n1, void* spec, long long sstride, int K2, const int* active,
                         const void* tw, const void* const* ge, const void* const* gs, const double* ih,
                         double halfvol, int n_rhs, cudaStream_t s);

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  typedef double2 type;
};
template <>
struct Cx<float> {
  typedef float2 type;
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}

// Batched Stockham FFT of `batch` sequences of length n stored contiguously in src (each
// sequence at offset b * n).  Uses dst as ping-pong buffer; returns the buffer holding the
// result.  tw[k] = exp(-2 pi i k / n) (shared memory).  INV selects exp(+...).
template <typename C, bool INV>
__device__ C* smem_fft(C* src, C* dst, const C* __restrict__ tw, const AxisPlan& ap, int batch) {
  const int n = ap.n;
  const int tid = threadIdx.x, nthr = blockDim.x;
  int Ns = 1;
  for (int st = 0; st < ap.nst; ++st) {
    const int R = ap.rad[st];
    const int nR = n / R;
    const int total = batch * nR;
    const int twstep = n / (Ns * R);
    for (int w = tid; w < total; w += nthr) {
      const int b = w / nR, j = w - b * nR;
      const C* in = src + b * n;
      C* out = dst + b * n;
      C v[5];
      for (int r = 0; r < R; ++r) v[r] = in[j + r * nR];
      const int jm = j % Ns;
      if (jm) {
        for (int r = 1; r < R; ++r) {
          const C t = tw[r * jm * twstep];
          v[r] = INV ? cmulc(v[r], t) : cmul(v[r], t);
        }
      }
      if (R == 2) {
        const C a = v[0], c = v[1];
        v[0] = cadd(a, c);
        v[1] = csub(a, c);
      } else if (R == 4) {
        const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
        C it3;  // -i t3 (forward) or +i t3 (inverse)
        if (INV) {
          it3.x = -t3.y;
          it3.y = t3.x;
        } else {
          it3.x = t3.y;
          it3.y = -t3.x;
        }
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, it3);
        v[3] = csub(t1, it3);
      } else {
        // generic small DFT (R = 3 or 5) with the table: y_k = sum_r v_r W_n^{(r k mod R) n/R}
        C y[5];
        const int s = n / R;
        for (int k = 0; k < R; ++k) {
          C acc = v[0];
          for (int r = 1; r < R; ++r) {
            const C t = tw[((r * k) % R) * s];
            acc = cadd(acc, INV ? cmulc(v[r], t) : cmul(v[r], t));
          }
          y[k] = acc;
        }
        for (int k = 0; k < R; ++k) v[k] = y[k];
      }
      const int base = (j / Ns) * Ns * R + jm;
      for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
    }
    __syncthreads();
    C* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

template <typename C>
__device__ __forceinline__ void load_tw(C* tws, const C* __restrict__ tw, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) tws[k] = tw[k];
}

// ---------------------------------------------------------------- pass 1: z, real -> complex
template <typename T>
__global__ void k_fft_z_r2c(T* __restrict__ f, typename Cx<T>::type* __restrict__ spec,
                            long long stride, long long sstride, AxisPlan ap, int K2, long long rows,
                            int pairs_per_block, const int* __restrict__ active,
                            const typename Cx<T>::type* __restrict__ tw,
                            unsigned long long* __restrict__ units, const T* __restrict__ q,
                            const RhsState* __restrict__ st) {
  typedef typename Cx<T>::type C;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  if (units && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(units, 1ULL);
  const int n = ap.n;
  C* tws = reinterpret_cast<C*>(smraw);
  C* b0 = tws + n;
  C* b1 = b0 + pairs_per_block * n;
  load_tw(tws, tw, n);
  const long long row0 = 2LL * blockIdx.x * pairs_per_block;
  const int nrows = (int)min((long long)2 * pairs_per_block, rows - row0);
  T* fr = f + rhs * stride + row0 * n;
  const T* qr = q ? q + rhs * stride + row0 * n : nullptr;
  const T alpha = q ? (T)st[rhs].alpha : T(0);
  for (int idx = threadIdx.x; idx < 2 * pairs_per_block * n; idx += blockDim.x) {
    const int rl = idx / n, k = idx - rl * n;
    T v = T(0);
    if (rl < nrows) {
      const long long o = (long long)rl * n + k;
      v = fr[o];
      if (q) {
        v -= alpha * qr[o];  // fused CG update f -= alpha A d
        fr[o] = v;
      }
    }
    T* dst = reinterpret_cast<T*>(&b0[(rl >> 1) * n + k]);
    dst[rl & 1] = v;
  }
  __syncthreads();
  C* res = smem_fft<C, false>(b0, b1, tws, ap, pairs_per_block);
  C* sp = spec + rhs * sstride + row0 * K2;
  for (int idx = threadIdx.x; idx < pairs_per_block * K2; idx += blockDim.x) {
    const int p = idx / K2, k = idx - p * K2;
    if (2 * p >= nrows) continue;
    const C zk = res[p * n + k];
    const C zn = res[p * n + (k == 0 ? 0 : n - k)];
    C X, Y;
    X.x = T(0.5) * (zk.x + zn.x);
    X.y = T(0.5) * (zk.y - zn.y);
    // Y = (zk - conj(zn)) / (2i)
    const T dx = zk.x - zn.x, dy = zk.y + zn.y;
    Y.x = T(0.5) * dy;
    Y.y = T(-0.5) * dx;
    sp[(long long)(2 * p) * K2 + k] = X;
    if (2 * p + 1 < nrows) sp[(long long)(2 * p + 1) * K2 + k] = Y;
  }
}

// ---------------------------------------------------------------- pass 2/4: y axis
template <typename T, bool INV>
__global__ void k_fft_y(typename Cx<T>::type* __restrict__ spec, long long sstride, AxisPlan ap,
                        int K2, int tk, int ntiles, const int* __restrict__ active,
                        const typename Cx<T>::type* __restrict__ tw) {
  typedef typename Cx<T>::type C;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int n = ap.n;  // = n1
  C* tws = reinterpret_cast<C*>(smraw);
  C* b0 = tws + n;
  C* b1 = b0 + tk * n;
  load_tw(tws, tw, n);
  const long long slab = blockIdx.x / ntiles;
  const int tile = blockIdx.x - (int)slab * ntiles;
  const int k0 = tile * tk;
  const int tke = min(tk, K2 - k0);
  C* sp = spec + rhs * sstride + slab * n * K2 + k0;
  for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
    const int j = idx / tk, kk = idx - j * tk;
    C v;
    v.x = T(0);
    v.y = T(0);
    if (kk < tke) v = sp[(long long)j * K2 + kk];
    b0[kk * n + j] = v;
  }
  __syncthreads();
  C* res = smem_fft<C, INV>(b0, b1, tws, ap, tk);
  for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
    const int j = idx / tk, kk = idx - j * tk;
    if (kk < tke) sp[(long long)j * K2 + kk] = res[kk * n + j];
  }
}

// ---------------------------------------------------------------- pass 3: x axis + Green
template <typename C, typename T>
__device__ __forceinline__ void green_solve(C& F0, C& F1, C& F2, C e0, C e1, C e2, C s0, C s1, C s2,
                                            T ih0, T ih1, T ih2, T halfvol) {
  // g_a = s_a / h_a
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
  if (!(S > T(0))) {
    F0.x = F0.y = F1.x = F1.y = F2.x = F2.y = T(0);
    return;
  }
  const C e[3] = {e0, e1, e2};
  C m01, m02, m12;
  m01.x = m01.y = m02.x = m02.y = m12.x = m12.y = T(0);
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
  // Cholesky M = L L^H, L lower with real diagonal; M(1,0) = conj(m01), M(2,0) = conj(m02),
  // M(2,1) = conj(m12)
  const T l00 = sqrt(d0);
  C l10, l20, l21;
  const T il00 = T(1) / l00;
  l10.x = m01.x * il00;
  l10.y = -m01.y * il00;
  l20.x = m02.x * il00;
  l20.y = -m02.y * il00;
  const T l11sq = d1 - (l10.x * l10.x + l10.y * l10.y);
  if (!(l11sq > T(0))) {
    F0.x = F0.y = F1.x = F1.y = F2.x = F2.y = T(0);
    return;
  }
  const T l11 = sqrt(l11sq);
  const T il11 = T(1) / l11;
  // l21 = (M(2,1) - l20 conj(l10)) / l11
  C m21;
  m21.x = m12.x;
  m21.y = -m12.y;
  const C t21 = csub(m21, cmulc(l20, l10));
  l21.x = t21.x * il11;
  l21.y = t21.y * il11;
  const T l22sq = d2 - (l20.x * l20.x + l20.y * l20.y) - (l21.x * l21.x + l21.y * l21.y);
  if (!(l22sq > T(0))) {
    F0.x = F0.y = F1.x = F1.y = F2.x = F2.y = T(0);
    return;
  }
  const T il22 = T(1) / sqrt(l22sq);
  // forward: L y = F
  C y0, y1, y2;
  y0.x = F0.x * il00;
  y0.y = F0.y * il00;
  C t = csub(F1, cmul(l10, y0));
  y1.x = t.x * il11;
  y1.y = t.y * il11;
  t = csub(csub(F2, cmul(l20, y0)), cmul(l21, y1));
  y2.x = t.x * il22;
  y2.y = t.y * il22;
  // backward: L^H x = y
  C x0, x1, x2;
  x2.x = y2.x * il22;
  x2.y = y2.y * il22;
  t = csub(y1, cmulc(x2, l21));  // conj(l21) * x2
  x1.x = t.x * il11;
  x1.y = t.y * il11;
  t = csub(csub(y0, cmulc(x1, l10)), cmulc(x2, l20));
  x0.x = t.x * il00;
  x0.y = t.y * il00;
  F0 = x0;
  F1 = x1;
  F2 = x2;
}

template <typename T>
__global__ void k_fft_x_green(typename Cx<T>::type* __restrict__ spec, long long sstride,
                              AxisPlan ap, int n1, int K2, int tk, int ntiles,
                              const int* __restrict__ active,
                              const typename Cx<T>::type* __restrict__ tw,
                              const typename Cx<T>::type* __restrict__ ge0,
                              const typename Cx<T>::type* __restrict__ ge1,
                              const typename Cx<T>::type* __restrict__ ge2,
                              const typename Cx<T>::type* __restrict__ gs0,
                              const typename Cx<T>::type* __restrict__ gs1,
                              const typename Cx<T>::type* __restrict__ gs2, T ih0, T ih1, T ih2,
                              T halfvol) {
  typedef typename Cx<T>::type C;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int n = ap.n;  // = n0
  C* tws = reinterpret_cast<C*>(smraw);
  C* b0 = tws + n;
  C* b1 = b0 + 3 * tk * n;
  load_tw(tws, tw, n);
  const int j = blockIdx.x / ntiles;
  const int tile = blockIdx.x - j * ntiles;
  const int k0 = tile * tk;
  const int tke = min(tk, K2 - k0);
  C* sp = spec + rhs * sstride;
  const long long cstride = (long long)n * n1 * K2;  // component stride
  const long long istride = (long long)n1 * K2;
  for (int idx = threadIdx.x; idx < 3 * n * tk; idx += blockDim.x) {
    const int ci = idx / tk, kk = idx - ci * tk;  // ci = c * n + i
    const int c = ci / n, i = ci - c * n;
    C v;
    v.x = T(0);
    v.y = T(0);
    if (kk < tke) v = sp[c * cstride + i * istride + (long long)j * K2 + k0 + kk];
    b0[(c * tk + kk) * n + i] = v;
  }
  __syncthreads();
  C* res = smem_fft<C, false>(b0, b1, tws, ap, 3 * tk);
  C* other = res == b0 ? b1 : b0;
  const C e1 = ge1[j], s1 = gs1[j];
  for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
    const int i = idx / tk, kk = idx - i * tk;
    if (kk >= tke) continue;
    C F0 = res[(0 * tk + kk) * n + i];
    C F1 = res[(1 * tk + kk) * n + i];
    C F2 = res[(2 * tk + kk) * n + i];
    green_solve<C, T>(F0, F1, F2, ge0[i], e1, ge2[k0 + kk], gs0[i], s1, gs2[k0 + kk], ih0, ih1, ih2,
                      halfvol);
    res[(0 * tk + kk) * n + i] = F0;
    res[(1 * tk + kk) * n + i] = F1;
    res[(2 * tk + kk) * n + i] = F2;
  }
  __syncthreads();
  C* out = smem_fft<C, true>(res, other, tws, ap, 3 * tk);
  for (int idx = threadIdx.x; idx < 3 * n * tk; idx += blockDim.x) {
    const int ci = idx / tk, kk = idx - ci * tk;
    const int c = ci / n, i = ci - c * n;
    if (kk < tke) sp[c * cstride + i * istride + (long long)j * K2 + k0 + kk] = out[(c * tk + kk) * n + i];
  }
}

// ---------------------------------------------------------------- pass 5: z, complex -> real
template <typename T>
__global__ void k_fft_z_c2r(const typename Cx<T>::type* __restrict__ spec, const T* __restrict__ f,
                            T* __restrict__ z, long long stride, long long sstride, AxisPlan ap,
                            int K2, long long rows, int pairs_per_block, T scale,
                            const int* __restrict__ active,
                            const typename Cx<T>::type* __restrict__ tw, double* __restrict__ partials,
                            int nparts) {
  typedef typename Cx<T>::type C;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int n = ap.n;
  C* tws = reinterpret_cast<C*>(smraw);
  C* b0 = tws + n;
  C* b1 = b0 + pairs_per_block * n;
  load_tw(tws, tw, n);
  const long long row0 = 2LL * blockIdx.x * pairs_per_block;
  const int nrows = (int)min((long long)2 * pairs_per_block, rows - row0);
  const C* sp = spec + rhs * sstride + row0 * K2;
  const int half = n / 2;
  for (int idx = threadIdx.x; idx < pairs_per_block * n; idx += blockDim.x) {
    const int p = idx / n, k = idx - p * n;
    C X, Y;
    X.x = X.y = Y.x = Y.y = T(0);
    if (2 * p < nrows) {
      const int kk = k <= half ? k : n - k;
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
    C Z;
    Z.x = X.x - Y.y;
    Z.y = X.y + Y.x;
    b0[p * n + k] = Z;
  }
  __syncthreads();
  C* res = smem_fft<C, true>(b0, b1, tws, ap, pairs_per_block);
  const T* fr = f + rhs * stride + row0 * n;
  T* zr = z + rhs * stride + row0 * n;
  double acc = 0.0;
  T tacc = T(0);
  for (int idx = threadIdx.x; idx < nrows * n; idx += blockDim.x) {
    const int rl = idx / n, k = idx - rl * n;
    const C v = res[(rl >> 1) * n + k];
    const T val = ((rl & 1) ? v.y : v.x) * scale;
    zr[(long long)rl * n + k] = val;
    tacc += val * fr[(long long)rl * n + k];
  }
  acc = (double)tacc;
  double vv[1] = {acc}, tot[1];
  block_sum<1>(vv, red, tot);
  if (threadIdx.x == 0) partials[(long long)rhs * nparts + blockIdx.x] = tot[0];
}

// ---------------------------------------------------------------- enriched block
// z_X = f_X (identity on the scaled enriched DOFs, eq. scaledPreconditioner) or, with eblk
// (6 x nX: inverse of each node's 3x3 block, entries 00, 11, 22, 01, 02, 12), z_X = B^-1 f_X per
// enriched node.  Enriched DOFs are component-major: f[off + c nX + j].
template <typename T>
__global__ void k_enr_precond(T* __restrict__ f, T* __restrict__ z, long long stride,
                              long long off, int nX, const int* __restrict__ active,
                              double* __restrict__ partials, int nparts, int slot0,
                              const T* __restrict__ q, const RhsState* __restrict__ st,
                              const T* __restrict__ eblk) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  T* fr = f + rhs * stride + off;
  T* zr = z + rhs * stride + off;
  const T* qr = q ? q + rhs * stride + off : nullptr;
  const T alpha = q ? (T)st[rhs].alpha : T(0);
  T acc = T(0);
  if (!eblk) {
    const long long count = 3LL * nX;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
      T v = fr[i];
      if (q) {
        v -= alpha * qr[i];  // fused CG update f -= alpha A d
        fr[i] = v;
      }
      zr[i] = v;
      acc += v * v;
    }
  } else {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nX; j += gridDim.x * blockDim.x) {
      T v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[c] = fr[(long long)c * nX + j];
        if (q) {
          v[c] -= alpha * qr[(long long)c * nX + j];
          fr[(long long)c * nX + j] = v[c];
        }
      }
      const T b00 = eblk[j], b11 = eblk[nX + j], b22 = eblk[2 * (long long)nX + j];
      const T b01 = eblk[3 * (long long)nX + j], b02 = eblk[4 * (long long)nX + j];
      const T b12 = eblk[5 * (long long)nX + j];
      const T z0 = b00 * v[0] + b01 * v[1] + b02 * v[2];
      const T z1 = b01 * v[0] + b11 * v[1] + b12 * v[2];
      const T z2 = b02 * v[0] + b12 * v[1] + b22 * v[2];
      zr[j] = z0;
      zr[nX + j] = z1;
      zr[2 * (long long)nX + j] = z2;
      acc += v[0] * z0 + v[1] * z1 + v[2] * z2;
    }
  }
  double vv[1] = {(double)acc}, tot[1];
  block_sum<1>(vv, red, tot);
  if (threadIdx.x == 0) partials[(long long)rhs * nparts + slot0 + blockIdx.x] = tot[0];
}

// ---------------------------------------------------------------- plan
static void factorize(int n, AxisPlan& ap) {
  ap.n = n;
  ap.nst = 0;
  int m = n;
  while (m % 4 == 0 && ap.nst < kMaxStages) {
    ap.rad[ap.nst++] = 4;
    m /= 4;
  }
  while (m % 2 == 0 && ap.nst < kMaxStages) {
    ap.rad[ap.nst++] = 2;
    m /= 2;
  }
  while (m % 3 == 0 && ap.nst < kMaxStages) {
    ap.rad[ap.nst++] = 3;
    m /= 3;
  }
  while (m % 5 == 0 && ap.nst < kMaxStages) {
    ap.rad[ap.nst++] = 5;
    m /= 5;
  }
  if (m != 1) ap.nst = -1;
}

static const int kFftThreads = 256;
static const size_t kSmemBudget = 96 * 1024;

static size_t smem_z(const FftPlan* p, size_t cs) { return cs * (p->n[2] + 2 * (size_t)p->xpairs * p->n[2]); }
static size_t smem_y(const FftPlan* p, size_t cs, int tk) { return cs * (p->n[1] + 2 * (size_t)tk * p->n[1]); }
static size_t smem_g(const FftPlan* p, size_t cs, int tk) { return cs * (p->n[0] + 6 * (size_t)tk * p->n[0]); }

FftPlan* fft_plan_create(const GridDev& g, cudaError_t* err) {
  *err = cudaSuccess;
  FftPlan* p = new FftPlan();
  p->g = g;
  p->n[0] = g.n0;
  p->n[1] = g.n1;
  p->n[2] = g.n2;
  p->K2 = g.n2 / 2 + 1;
  p->fast = fast_fft_supported(g.n0) && fast_fft_supported(g.n1) && fast_fft_supported(g.n2) &&
            true;
  for (int a = 0; a < 3; ++a) {
    factorize(p->n[a], p->ax[a]);
    if (p->ax[a].nst < 0) {
      *err = cudaErrorInvalidValue;
      delete p;
      return nullptr;
    }
  }
  // tiles: z passes process `xpairs` row pairs per block; the y pass a k2 tile of width ytk;
  // the Green pass a k2 tile sized to the shared-memory budget
  p->xpairs = 8;
  while (p->xpairs > 1 && 16 * (size_t)(p->n[2] + 2 * p->xpairs * p->n[2]) > kSmemBudget) p->xpairs /= 2;
  for (int prec = 0; prec < 2; ++prec) {
    const size_t cs = prec == 0 ? 16 : 8;
    int tkmax = 16;
    while (tkmax > 1 && smem_y(p, cs, tkmax) > kSmemBudget) --tkmax;
    const int nt = (p->K2 + tkmax - 1) / tkmax;
    const int tk = (p->K2 + nt - 1) / nt;
    if (prec == 0) {
      p->ytk_d = tk;
      p->ytiles_d = nt;
    } else {
      p->ytk_f = tk;
      p->ytiles_f = nt;
    }
  }
  for (int prec = 0; prec < 2; ++prec) {
    const size_t cs = prec == 0 ? 16 : 8;
    int tkmax = 16;
    while (tkmax > 1 && smem_g(p, cs, tkmax) > kSmemBudget) --tkmax;
    const int nt = (p->K2 + tkmax - 1) / tkmax;
    const int tk = (p->K2 + nt - 1) / nt;
    if (prec == 0) {
      p->gtk_d = tk;
      p->gtiles_d = nt;
    } else {
      p->gtk_f = tk;
      p->gtiles_f = nt;
    }
  }
  // tables: twiddles exp(-2 pi i k / n) and Green phases per axis
  size_t tot2d = 0;
  for (int a = 0; a < 3; ++a) tot2d += 3 * (size_t)p->n[a];
  void* pool = nullptr;
  *err = cudaMalloc(&pool, tot2d * (sizeof(double2) + sizeof(float2)));
  if (*err != cudaSuccess) {
    delete p;
    return nullptr;
  }
  p->pool = pool;
  std::vector<double2> hd(tot2d);
  std::vector<float2> hf(tot2d);
  size_t off = 0;
  double2* dbase = reinterpret_cast<double2*>(pool);
  float2* fbase = reinterpret_cast<float2*>(dbase + tot2d);
  for (int a = 0; a < 3; ++a) {
    const int n = p->n[a];
    p->twd[a] = dbase + off;
    p->twf[a] = fbase + off;
    p->ged[a] = dbase + off + n;
    p->gef[a] = fbase + off + n;
    p->gsd[a] = dbase + off + 2 * n;
    p->gsf[a] = fbase + off + 2 * n;
    for (int k = 0; k < n; ++k) {
      const double th = 2.0 * M_PI * (double)k / (double)n;
      const double c = cos(th), s = sin(th), sh = sin(0.5 * th);
      hd[off + k] = make_double2(c, -s);
      hd[off + n + k] = make_double2(c, s);
      hd[off + 2 * n + k] = make_double2(-2.0 * sh * sh, s);
    }
    off += 3 * n;
  }
  for (size_t i = 0; i < tot2d; ++i) hf[i] = make_float2((float)hd[i].x, (float)hd[i].y);
  *err = cudaMemcpy(dbase, hd.data(), tot2d * sizeof(double2), cudaMemcpyHostToDevice);
  if (*err == cudaSuccess)
    *err = cudaMemcpy(fbase, hf.data(), tot2d * sizeof(float2), cudaMemcpyHostToDevice);
  if (*err != cudaSuccess) {
    cudaFree(pool);
    delete p;
    return nullptr;
  }
  // opt in to the largest dynamic shared memory size any pass uses
  size_t need = 0;
  for (int prec = 0; prec < 2; ++prec) {
    const size_t cs = prec == 0 ? 16 : 8;
    need = std::max(need, smem_z(p, cs));
    need = std::max(need, smem_y(p, cs, prec == 0 ? p->ytk_d : p->ytk_f));
    need = std::max(need, smem_g(p, cs, prec == 0 ? p->gtk_d : p->gtk_f));
  }
  if (need > 227 * 1024) {
    *err = cudaErrorInvalidValue;
    cudaFree(pool);
    delete p;
    return nullptr;
  }
  // slab path: Green factor table (depends on the grid only)
  p->slab = false;
  p->gtab = nullptr;
  if (p->fast && slab_supported(g.n0, g.n1, g.n2)) {
    *err = cudaMalloc(&p->gtab, slab_table_floats(g.n0, g.n1) * sizeof(float));
    if (*err == cudaSuccess) {
      const void* ge[3] = {p->gef[0], p->gef[1], p->gef[2]};
      const void* gs[3] = {p->gsf[0], p->gsf[1], p->gsf[2]};
      const double ih[3] = {1.0 / g.h[0], 1.0 / g.h[1], 1.0 / g.h[2]};
      *err = slab_green_table(p->gtab, g.n0, g.n1, ge, gs, ih, 0.5 * g.vol_tet, 0);
      if (*err == cudaSuccess) *err = cudaDeviceSynchronize();
    }
    if (*err != cudaSuccess) {
      if (p->gtab) cudaFree(p->gtab);
      cudaFree(pool);
      delete p;
      return nullptr;
    }
    p->slab = true;
  }
  const int big = (int)need;
  cudaFuncSetAttribute(k_fft_z_r2c<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_z_r2c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_z_c2r<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_z_c2r<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_y<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_y<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_y<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_y<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_x_green<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_fft_x_green<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  *err = cudaGetLastError();
  return p;
}

void fft_plan_destroy(FftPlan* p) {
  if (!p) return;
  if (p->pool) cudaFree(p->pool);
  if (p->gtab) cudaFree(p->gtab);
  delete p;
}

size_t fft_spectrum_elems(const FftPlan* p) { return 3ULL * p->n[0] * p->n[1] * p->K2; }

static int zpass_blocks(const FftPlan* p, bool dbl) {
  if (p->slab && !dbl) return slab_z_blocks(p->n[0]);
  if (p->fast) return fast_z_blocks(p->n[0], p->n[1], p->n[2]);
  const long long rows = 3LL * p->n[0] * p->n[1];
  return (int)((rows + 2LL * p->xpairs - 1) / (2LL * p->xpairs));
}

static int enr_blocks(int nX) {
  if (nX <= 0) return 1;
  const long long n = 3LL * nX;
  long long nb = (n + 255) / 256;
  if (nb > 256) nb = 256;
  return (int)nb;
}

int precondition_blocks(const FftPlan* p, int nX, bool dbl) { return zpass_blocks(p, dbl) + enr_blocks(nX); }

template <typename T>
cudaError_t launch_precondition(const FftPlan* p, T* f, T* z, void* spec_v, long long stride,
                                int nX, const int* active, double* partials, int nparts,
                                int n_rhs, cudaStream_t s, unsigned long long* units, const T* q,
                                const RhsState* st, const T* eblk, int group) {
  // nX < 0: the standard part only (a group of a grouped call; the caller does the enriched part)
  typedef typename Cx<T>::type C;
  const bool dbl0 = sizeof(T) == 8;
  if (group > 0 && group < n_rhs && (p->slab || p->fast) && !(p->slab && !p->fast && dbl0)) {
    // the three (or five) FFT passes for `group` right-hand sides at a time: the spectrum of a
    // group can stay in L2 between the passes; the enriched block afterwards for all of them
    const int zb = zpass_blocks(p, dbl0);
    const bool use_slab = p->slab && !dbl0;
    for (int r0 = 0; r0 < n_rhs; r0 += group) {
      const int nr = n_rhs - r0 < group ? n_rhs - r0 : group;
      cudaError_t e = launch_precondition<T>(p, f + r0 * stride, z + r0 * stride, spec_v, stride, -1,
                                             active ? active + r0 : nullptr, partials + (long long)r0 * nparts,
                                             nparts, nr, s, units, q ? q + r0 * stride : nullptr,
                                             st ? st + r0 : nullptr, nullptr, 0);
      if (e != cudaSuccess) return e;
    }
    (void)use_slab;
    k_enr_precond<T><<<dim3(enr_blocks(nX), n_rhs), 256, 0, s>>>(f, z, stride, 3 * p->g.N, nX, active,
                                                                 partials, nparts, zb, q, st, eblk);
    return cudaGetLastError();
  }
  const bool dbl = sizeof(T) == 8;
  const int a2 = 2;  // z axis
  C* spec = reinterpret_cast<C*>(spec_v);
  const long long sstride = (long long)fft_spectrum_elems(p);
  const long long rows = 3LL * p->n[0] * p->n[1];
  const size_t cs = sizeof(C);
  const C* tw0 = reinterpret_cast<const C*>(dbl ? (const void*)p->twd[0] : (const void*)p->twf[0]);
  const C* tw1 = reinterpret_cast<const C*>(dbl ? (const void*)p->twd[1] : (const void*)p->twf[1]);
  const C* tw2 = reinterpret_cast<const C*>(dbl ? (const void*)p->twd[a2] : (const void*)p->twf[a2]);
  const int zb = zpass_blocks(p, dbl);
  if (p->slab && !dbl) {
    const void* ge[3] = {p->gef[0], p->gef[1], p->gef[2]};
    const void* gs[3] = {p->gsf[0], p->gsf[1], p->gsf[2]};
    const double ih[3] = {1.0 / p->g.h[0], 1.0 / p->g.h[1], 1.0 / p->g.h[2]};
    cudaError_t e = slab_precondition(p->n[0], p->n[1], (float*)f, (float*)z, spec, stride, sstride, active, p->twf[0],
                                      p->twf[1], p->twf[2], p->gtab, ge, gs, ih, 0.5 * p->g.vol_tet, units,
                                      (const float*)q, st, partials, nparts, n_rhs, s);
    if (e != cudaSuccess) return e;
    if (nX >= 0) k_enr_precond<T><<<dim3(enr_blocks(nX), n_rhs), 256, 0, s>>>(f, z, stride, 3 * p->g.N, nX, active,
                                                                 partials, nparts, zb, q, st, eblk);
    return cudaGetLastError();
  }
  if (p->fast) {
    const void* ge[3];
    const void* gs[3];
    for (int a = 0; a < 3; ++a) {
      ge[a] = dbl ? (const void*)p->ged[a] : (const void*)p->gef[a];
      gs[a] = dbl ? (const void*)p->gsd[a] : (const void*)p->gsf[a];
    }
    const double ih[3] = {1.0 / p->g.h[0], 1.0 / p->g.h[1], 1.0 / p->g.h[2]};
    cudaError_t e = fast_z_r2c<T>(p->n[2], f, spec, stride, sstride, p->n[0], p->n[1], active, tw2, units,
                                  n_rhs, s, q, st);
    if (e == cudaSuccess) e = fast_y<T, false>(p->n[1], p->n[0], spec, sstride, p->K2, active, tw1, n_rhs, s);
    if (e == cudaSuccess)
      e = fast_x_green<T>(p->n[0], p->n[1], spec, sstride, p->K2, active, tw0, ge, gs, ih, 0.5 * p->g.vol_tet,
                          n_rhs, s);
    if (e == cudaSuccess) e = fast_y<T, true>(p->n[1], p->n[0], spec, sstride, p->K2, active, tw1, n_rhs, s);
    if (e == cudaSuccess)
      e = fast_z_c2r<T>(p->n[2], spec, f, z, stride, sstride, p->n[0], p->n[1],
                        1.0 / ((double)p->n[0] * p->n[1] * p->n[2]), active, tw2, partials, nparts, n_rhs, s);
    if (e != cudaSuccess) return e;
    if (nX >= 0) k_enr_precond<T><<<dim3(enr_blocks(nX), n_rhs), 256, 0, s>>>(f, z, stride, 3 * p->g.N, nX, active,
                                                                 partials, nparts, zb, q, st, eblk);
    return cudaGetLastError();
  }
  k_fft_z_r2c<T><<<dim3(zb, n_rhs), kFftThreads, smem_z(p, cs), s>>>(
      f, spec, stride, sstride, p->ax[2], p->K2, rows, p->xpairs, active, tw2, units, q, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ytk = dbl ? p->ytk_d : p->ytk_f;
  const int ytiles = dbl ? p->ytiles_d : p->ytiles_f;
  const int yb = p->n[0] * 3 * ytiles;
  k_fft_y<T, false><<<dim3(yb, n_rhs), kFftThreads, smem_y(p, cs, ytk), s>>>(
      spec, sstride, p->ax[1], p->K2, ytk, ytiles, active, tw1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int gtk = dbl ? p->gtk_d : p->gtk_f;
  const int gtiles = dbl ? p->gtiles_d : p->gtiles_f;
  const C* ge[3];
  const C* gs[3];
  for (int a = 0; a < 3; ++a) {
    ge[a] = reinterpret_cast<const C*>(dbl ? (const void*)p->ged[a] : (const void*)p->gef[a]);
    gs[a] = reinterpret_cast<const C*>(dbl ? (const void*)p->gsd[a] : (const void*)p->gsf[a]);
  }
  const GridDev& g = p->g;
  k_fft_x_green<T><<<dim3(p->n[1] * gtiles, n_rhs), kFftThreads, smem_g(p, cs, gtk), s>>>(
      spec, sstride, p->ax[0], p->n[1], p->K2, gtk, gtiles, active, tw0, ge[0], ge[1], ge[2], gs[0],
      gs[1], gs[2], (T)(1.0 / g.h[0]), (T)(1.0 / g.h[1]), (T)(1.0 / g.h[2]), (T)(0.5 * g.vol_tet));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fft_y<T, true><<<dim3(yb, n_rhs), kFftThreads, smem_y(p, cs, ytk), s>>>(
      spec, sstride, p->ax[1], p->K2, ytk, ytiles, active, tw1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const T scale = (T)(1.0 / ((double)p->n[0] * p->n[1] * p->n[2]));
  k_fft_z_c2r<T><<<dim3(zb, n_rhs), kFftThreads, smem_z(p, cs), s>>>(
      spec, f, z, stride, sstride, p->ax[2], p->K2, rows, p->xpairs, scale, active, tw2, partials,
      nparts);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long N = g.N;
  if (nX >= 0) k_enr_precond<T><<<dim3(enr_blocks(nX), n_rhs), 256, 0, s>>>(f, z, stride, 3 * N, nX, active,
                                                                 partials, nparts, zb, q, st, eblk);
  return cudaGetLastError();
}

template cudaError_t launch_precondition<float>(const FftPlan*, float*, float*, void*, long long, int,
                                                const int*, double*, int, int, cudaStream_t,
                                                unsigned long long*, const float*, const RhsState*,
                                                const float*, int);
template cudaError_t launch_precondition<double>(const FftPlan*, double*, double*, void*, long long, int,
                                                 const int*, double*, int, int, cudaStream_t,
                                                 unsigned long long*, const double*, const RhsState*,
                                                 const double*, int);

}  // namespace xfft
