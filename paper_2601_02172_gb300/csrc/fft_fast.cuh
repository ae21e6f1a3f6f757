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
XFFT_PLAN(384, 24, 8, 8, 2, 3)
#undef XFFT_PLAN

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
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV>
__device__ __forceinline__ C mul_mi(C a) {
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
  __device__ __forceinline__ static void run(C* v) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C, bool INV>
struct Dft<C, 4, INV> {
  __device__ __forceinline__ static void run(C* v) {
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
  __device__ __forceinline__ static void run(C* v) {
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
  __device__ __forceinline__ static void run(C* v) {
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

// radix 8 = two radix-4 DFTs on even / odd inputs combined with W8^k
template <typename C, bool INV>
struct Dft<C, 8, INV> {
  __device__ __forceinline__ static void run(C* v) {
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

template <typename C, bool INV>
struct Dft<C, 1, INV> {
  __device__ __forceinline__ static void run(C*) {}
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

}  // namespace fast
}  // namespace xfft
