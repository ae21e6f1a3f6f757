// Host build of the CUDA path's radix butterflies (the in-register DFTs of the Stockham FFT
// stages), for the CPU test against a direct DFT.
#include "fft_fast.cuh"

namespace {
template <int R, bool INV>
void run(double* v) {
  double2 c[R > 1 ? R : 1];
  for (int k = 0; k < R; ++k) c[k] = make_double2(v[2 * k], v[2 * k + 1]);
  xfft::fast::Dft<double2, R, INV>::run(c);
  for (int k = 0; k < R; ++k) {
    v[2 * k] = c[k].x;
    v[2 * k + 1] = c[k].y;
  }
}
}  // namespace

// v: R complex values (interleaved re, im), transformed in place; returns 0 for an unknown radix
extern "C" int host_dft(int R, int inv, double* v) {
  switch (R) {
    case 2: inv ? run<2, true>(v) : run<2, false>(v); return 1;
    case 3: inv ? run<3, true>(v) : run<3, false>(v); return 1;
    case 4: inv ? run<4, true>(v) : run<4, false>(v); return 1;
    case 5: inv ? run<5, true>(v) : run<5, false>(v); return 1;
    case 6: inv ? run<6, true>(v) : run<6, false>(v); return 1;
    case 8: inv ? run<8, true>(v) : run<8, false>(v); return 1;
    case 16: inv ? run<16, true>(v) : run<16, false>(v); return 1;
    default: return 0;
  }
}
