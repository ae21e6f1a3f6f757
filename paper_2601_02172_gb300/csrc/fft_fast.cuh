// Compile-time planned line FFTs for the X-FFT preconditioner.
//
// A line of length N lives in shared memory; T = N / E threads cooperate on it, each holding E
// complex values in registers.  Each Stockham stage of radix R (R divides E) is done in place:
// every thread loads its E/R butterflies' inputs, the block synchronises, the butterflies run
// in registers (twiddles from a shared table), and the outputs are stored in sorted order.
// The radix sequence and E are fixed per length at compile time, so all index arithmetic is by
// constants.
#pragma once

#include <cuda_runtime.h>

#include "xfft_common.cuh"

namespace xfft {
namespace fast {

// Plan per length: elements per thread E and up to four radices (1 = unused)
template <int N>
struct Plan {
  static constexpr bool ok = false;
};
#define XFFT_PLAN(n, e, r0, r1, r2, r3)                                     \
  template <>                                                               \
  struct Plan<n> {                                                          \
    static constexpr bool ok = true;                                        \
    static constexpr int E = e;                                             \
    static constexpr int R0 = r0, R1 = r1, R2 = r2, R3 = r3;                \
  };
XFFT_PLAN(16, 4, 4, 4, 1, 1)
XFFT_PLAN(32, 8, 8, 4, 1, 1)
XFFT_PLAN(48, 12, 4, 4, 3, 1)
XFFT_PLAN(64, 8, 8, 8, 1, 1)
XFFT_PLAN(80, 20, 4, 4, 5, 1)
XFFT_PLAN(96, 12, 4, 4, 2, 3)
XFFT_PLAN(128, 8, 8, 8, 2, 1)
XFFT_PLAN(192, 24, 8, 8, 3, 1)
XFFT_PLAN(256, 8, 8, 8, 4, 1)
XFFT_PLAN(384, 12, 4, 4, 4, 6)
#undef XFFT_PLAN
// radix sequence for E elements per thread (the default plan, or fewer passes where E allows)
template <int N, int E>
struct PlanE {
  static constexpr int R0 = Plan<N>::R0, R1 = Plan<N>::R1, R2 = Plan<N>::R2, R3 = Plan<N>::R3;
};
template <>
struct PlanE<128, 16> {
  static constexpr int R0 = 16, R1 = 8, R2 = 1, R3 = 1;
};
// every length with a plan (host-side dispatch lists)
#define XFFT_FAST_SIZES(X) X(16) X(32) X(48) X(64) X(80) X(96) X(128) X(192) X(256) X(384)

template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__host__ __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename C>
__host__ __device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename C>
__host__ __device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV>
__host__ __device__ __forceinline__ C mul_mi(C a) {
  C r;
  if (INV) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}

// ---------------------------------------------------------------- radix butterflies
template <typename C, int R, bool INV>
struct Dft;

template <typename C, bool INV>
struct Dft<C, 2, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C, bool INV>
struct Dft<C, 4, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const C t2 = cadd(v[1], v[3]), t3 = mul_mi<C, INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

// y_k = sum_r v_r exp(-+2 pi i r k / 3):  with s = sin(2 pi / 3)
template <typename C, bool INV>
struct Dft<C, 3, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    typedef decltype(v[0].x) T;
    const T s = (T)0.86602540378443864676;  // sqrt(3) / 2
    const C t1 = cadd(v[1], v[2]);
    C m;  // a - (b + c) / 2
    m.x = v[0].x - (T)0.5 * t1.x;
    m.y = v[0].y - (T)0.5 * t1.y;
    C d = csub(v[1], v[2]);
    d.x *= s;
    d.y *= s;
    const C id = mul_mi<C, INV>(d);  // -i s (b - c) forward
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, id);
    v[2] = csub(m, id);
  }
};

// radix 5 with c1 = cos(2 pi/5), c2 = cos(4 pi/5), s1 = sin(2 pi/5), s2 = sin(4 pi/5)
template <typename C, bool INV>
struct Dft<C, 5, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    typedef decltype(v[0].x) T;
    const T c1 = (T)0.30901699437494742410;   // (sqrt5 - 1) / 4
    const T c2 = (T)-0.80901699437494742410;  // -(sqrt5 + 1) / 4
    const T s1 = (T)0.95105651629515357212;   // sqrt((5 + sqrt5) / 8)
    const T s2 = (T)0.58778525229247312917;   // sqrt((5 - sqrt5) / 8)
    const C p14 = cadd(v[1], v[4]), m14 = csub(v[1], v[4]);
    const C p23 = cadd(v[2], v[3]), m23 = csub(v[2], v[3]);
    C a1, a2, b1, b2;
    a1.x = v[0].x + c1 * p14.x + c2 * p23.x;
    a1.y = v[0].y + c1 * p14.y + c2 * p23.y;
    a2.x = v[0].x + c2 * p14.x + c1 * p23.x;
    a2.y = v[0].y + c2 * p14.y + c1 * p23.y;
    b1.x = s1 * m14.x + s2 * m23.x;
    b1.y = s1 * m14.y + s2 * m23.y;
    b2.x = s2 * m14.x - s1 * m23.x;
    b2.y = s2 * m14.y - s1 * m23.y;
    const C ib1 = mul_mi<C, INV>(b1), ib2 = mul_mi<C, INV>(b2);
    v[0] = cadd(v[0], cadd(p14, p23));
    v[1] = cadd(a1, ib1);
    v[4] = csub(a1, ib1);
    v[2] = cadd(a2, ib2);
    v[3] = csub(a2, ib2);
  }
};

// radix 6 = two radix-3 DFTs on even / odd inputs combined with W6^k: X_k = E_k + W6^k O_k,
// X_{k+3} = E_k - W6^k O_k (k < 3), W6 = exp(-+2 pi i / 6) = 1/2 -+ i sqrt(3)/2
template <typename C, bool INV>
struct Dft<C, 6, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    typedef decltype(v[0].x) T;
    const T h = (T)0.5, s = INV ? (T)0.86602540378443864676 : (T)-0.86602540378443864676;
    C e[3] = {v[0], v[2], v[4]};
    C o[3] = {v[1], v[3], v[5]};
    Dft<C, 3, INV>::run(e);
    Dft<C, 3, INV>::run(o);
    C w1, w2;  // W6^1 o_1 = (h + i s) o_1, W6^2 o_2 = (-h + i s) o_2
    w1.x = h * o[1].x - s * o[1].y;
    w1.y = h * o[1].y + s * o[1].x;
    w2.x = -h * o[2].x - s * o[2].y;
    w2.y = -h * o[2].y + s * o[2].x;
    v[0] = cadd(e[0], o[0]);
    v[3] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[4] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[5] = csub(e[2], w2);
  }
};

// radix 8 = two radix-4 DFTs on even / odd inputs combined with W8^k
template <typename C, bool INV>
struct Dft<C, 8, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    typedef decltype(v[0].x) T;
    const T r = (T)0.70710678118654752440;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<C, 4, INV>::run(e);
    Dft<C, 4, INV>::run(o);
    // W8^1 = (1 - i)/sqrt2 forward, (1 + i)/sqrt2 inverse; W8^2 = -+i; W8^3 = (-1 -+ i)/sqrt2
    C w1, w3;
    if (INV) {
      w1.x = r * (o[1].x - o[1].y);
      w1.y = r * (o[1].x + o[1].y);
      w3.x = -r * (o[3].x + o[3].y);
      w3.y = r * (o[3].x - o[3].y);
    } else {
      w1.x = r * (o[1].x + o[1].y);
      w1.y = r * (o[1].y - o[1].x);
      w3.x = r * (o[3].y - o[3].x);
      w3.y = -r * (o[3].x + o[3].y);
    }
    const C w2 = mul_mi<C, INV>(o[2]);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);
    v[7] = csub(e[3], w3);
  }
};

// radix 16 = 4 x 4: inputs n = 4a + b, outputs k = c + 4d; DFT4 over a, twiddle W16^(b c),
// DFT4 over b.  c1 = cos(pi/8), s1 = sin(pi/8)
template <typename C, bool INV>
struct Dft<C, 16, INV> {
  __host__ __device__ __forceinline__ static void run(C* v) {
    typedef decltype(v[0].x) T;
    const T c1 = (T)0.92387953251128675613;
    const T s1 = (T)0.38268343236508977173;
    const T r = (T)0.70710678118654752440;
    const T sg = INV ? T(1) : T(-1);  // sign of the imaginary part of W16^1
    C y[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      C t[4] = {v[b], v[b + 4], v[b + 8], v[b + 12]};
      Dft<C, 4, INV>::run(t);
#pragma unroll
      for (int c = 0; c < 4; ++c) y[b][c] = t[c];
    }
    C w1, w2, w3, w6, w9;
    w1.x = c1;
    w1.y = sg * s1;
    w2.x = r;
    w2.y = sg * r;
    w3.x = s1;
    w3.y = sg * c1;
    w6.x = -r;
    w6.y = sg * r;
    w9.x = -c1;
    w9.y = -sg * s1;
    y[1][1] = cmul(y[1][1], w1);
    y[1][2] = cmul(y[1][2], w2);
    y[1][3] = cmul(y[1][3], w3);
    y[2][1] = cmul(y[2][1], w2);
    y[2][2] = mul_mi<C, INV>(y[2][2]);  // W16^4 = -+i
    y[2][3] = cmul(y[2][3], w6);
    y[3][1] = cmul(y[3][1], w3);
    y[3][2] = cmul(y[3][2], w6);
    y[3][3] = cmul(y[3][3], w9);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      C t[4] = {y[0][c], y[1][c], y[2][c], y[3][c]};
      Dft<C, 4, INV>::run(t);
#pragma unroll
      for (int d = 0; d < 4; ++d) v[c + 4 * d] = t[d];
    }
  }
};

template <typename C, bool INV>
struct Dft<C, 1, INV> {
  __host__ __device__ __forceinline__ static void run(C*) {}
};

// One in-place Stockham stage of radix R on a line (stride-1 elements at `line`), thread t of
// the line's T = N / E threads.  NS = product of the previous radices.  tw[k] = exp(-2 pi i k/N).
template <typename C, int N, int E, int R, int NS, bool INV>
__device__ __forceinline__ void stage(C* line, const C* __restrict__ tw, int t) {
  if (R == 1) return;
  constexpr int T = N / E;
  constexpr int NR = N / R;
  constexpr int BPT = E / R;
  C v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = t + b * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = line[j + r * NR];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = t + b * T;
    const int jm = j % NS;
    if (NS > 1) {
      constexpr int step = N / (NS * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C w = tw[r * jm * step];
        v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
      }
    }
    Dft<C, R, INV>::run(v[b]);
    const int base = (j / NS) * NS * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) line[base + r * NS] = v[b][r];
  }
  __syncthreads();
}

// Full line transform (all threads of the block must call it; t < N/E selects the thread's
// position in its line, lines beyond the data may run on dummy storage).
template <typename C, int N, bool INV>
__device__ __forceinline__ void line_fft(C* line, const C* __restrict__ tw, int t) {
  typedef Plan<N> P;
  constexpr int E = P::E;
  constexpr int N0 = 1, N1 = P::R0, N2 = P::R0 * P::R1, N3 = P::R0 * P::R1 * P::R2;
  stage<C, N, E, P::R0, N0, INV>(line, tw, t);
  stage<C, N, E, P::R1, N1, INV>(line, tw, t);
  stage<C, N, E, P::R2, N2, INV>(line, tw, t);
  stage<C, N, E, P::R3, N3, INV>(line, tw, t);
}

// ---------------------------------------------------------------- Green operator
// Cholesky factor of M(xi) = (|T|/2) sum_tets (|G|^2 I + G G^H) (see fft.cu); returns false
// at xi = 0 or on a non-positive pivot (the Green operator then maps to 0).  Host and device
// (the host build is checked against the oracle's symbol on the CPU).
template <typename C, typename T>
struct GreenFactor {
  T il00, il11, il22;
  C l10, l20, l21;
};

template <typename C, typename T>
__host__ __device__ __forceinline__ bool green_factor(GreenFactor<C, T>& gf, C e0, C e1, C e2, C s0, C s1,
                                                      C s2, T ih0, T ih1, T ih2, T halfvol) {
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
  if (!(S > T(0))) return false;
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
  // M = L L^H with M(1,0) = conj(m01), M(2,0) = conj(m02), M(2,1) = conj(m12)
  gf.il00 = T(1) / sqrt(d0);
  gf.l10.x = m01.x * gf.il00;
  gf.l10.y = -m01.y * gf.il00;
  gf.l20.x = m02.x * gf.il00;
  gf.l20.y = -m02.y * gf.il00;
  const T l11sq = d1 - (gf.l10.x * gf.l10.x + gf.l10.y * gf.l10.y);
  if (!(l11sq > T(0))) return false;
  gf.il11 = T(1) / sqrt(l11sq);
  C m21;
  m21.x = m12.x;
  m21.y = -m12.y;
  const C t21 = csub(m21, cmulc(gf.l20, gf.l10));
  gf.l21.x = t21.x * gf.il11;
  gf.l21.y = t21.y * gf.il11;
  const T l22sq = d2 - (gf.l20.x * gf.l20.x + gf.l20.y * gf.l20.y) - (gf.l21.x * gf.l21.x + gf.l21.y * gf.l21.y);
  if (!(l22sq > T(0))) return false;
  gf.il22 = T(1) / sqrt(l22sq);
  return true;
}

template <typename C, typename T>
__host__ __device__ __forceinline__ void green_solve(const GreenFactor<C, T>& gf, C& F0, C& F1, C& F2) {
  C y0, y1, y2, t;
  y0.x = F0.x * gf.il00;
  y0.y = F0.y * gf.il00;
  t = csub(F1, cmul(gf.l10, y0));
  y1.x = t.x * gf.il11;
  y1.y = t.y * gf.il11;
  t = csub(csub(F2, cmul(gf.l20, y0)), cmul(gf.l21, y1));
  y2.x = t.x * gf.il22;
  y2.y = t.y * gf.il22;
  C x0, x1, x2;
  x2.x = y2.x * gf.il22;
  x2.y = y2.y * gf.il22;
  t = csub(y1, cmulc(x2, gf.l21));
  x1.x = t.x * gf.il11;
  x1.y = t.y * gf.il11;
  t = csub(csub(y0, cmulc(x1, gf.l10)), cmulc(x2, gf.l20));
  x0.x = t.x * gf.il00;
  x0.y = t.y * gf.il00;
  F0 = x0;
  F1 = x1;
  F2 = x2;
}

// block: (k2, j), all three components of a group of rg right-hand sides: 3 rg contiguous lines
// of length N = n0.  The symbol of each frequency is factorised once and applied to every
// right-hand side of the group.

// ---------------------------------------------------------------- lines with an address map
// The same stages on a line whose element m lives at map.at(m) (any shared-memory layout; the
// maps of different lines must be disjoint).  The first stage may read its inputs through a
// different map `ld0` (ld0.get(m) returns the value).  Threads with act == false take part in
// the barriers only.
template <typename C, int N, int E, int R, int NS, bool INV, class LD, class MAP>
__device__ __forceinline__ void stage_map(const LD& ld, const MAP& mp, const C* __restrict__ tw, int t,
                                          bool act) {
  if (R == 1) return;
  constexpr int T = N / E;
  constexpr int NR = N / R;
  constexpr int BPT = E / R;
  C v[BPT][R];
  if (act) {
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
      const int j = t + b * T;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = ld.get(j + r * NR);
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
      const int j = t + b * T;
      const int jm = j % NS;
      if (NS > 1) {
        constexpr int step = N / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C w = tw[r * jm * step];
          v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
        }
      }
      Dft<C, R, INV>::run(v[b]);
      const int base = (j / NS) * NS * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) *mp.at(base + r * NS) = v[b][r];
    }
  }
  __syncthreads();
}

template <typename C, class MAP>
struct MapLoad {  // reads through the line's own map
  const MAP& m;
  __device__ __forceinline__ C get(int k) const { return *m.at(k); }
};

// Line transform with E elements per thread (E divisible by every radix of Plan<N>).
template <typename C, int N, int E, bool INV, class LD0, class MAP>
__device__ __forceinline__ void line_fft_map(const LD0& ld0, const MAP& mp, const C* __restrict__ tw, int t,
                                             bool act) {
  typedef PlanE<N, E> P;
  static_assert(E % P::R0 == 0 && E % P::R1 == 0 && E % P::R2 == 0 && E % P::R3 == 0, "E vs radices");
  constexpr int N1 = P::R0, N2 = P::R0 * P::R1, N3 = P::R0 * P::R1 * P::R2;
  const MapLoad<C, MAP> ld{mp};
  stage_map<C, N, E, P::R0, 1, INV>(ld0, mp, tw, t, act);
  stage_map<C, N, E, P::R1, N1, INV>(ld, mp, tw, t, act);
  stage_map<C, N, E, P::R2, N2, INV>(ld, mp, tw, t, act);
  stage_map<C, N, E, P::R3, N3, INV>(ld, mp, tw, t, act);
}

}  // namespace fast
}  // namespace xfft
