// Host side of the slab path (kernels and launchers in fft_slab.cuh): which grids it serves, its
// Green factor table and the dispatch on the plane size.  The 128 x 128 launchers are
// instantiated here, the smaller plane sizes in fft_slab_sq.cu.
#include "fft_slab.cuh"

namespace xfft {
namespace slab {
XFFT_SLAB_INST(128)
XFFT_SLAB_SMALL(XFFT_SLAB_DECL)
}  // namespace slab

static bool slab_plane(int n1) {
  switch (n1) {
#define X(n) case n:
    XFFT_SLAB_SMALL(X)
#undef X
    case 128:
      return true;
    default:
      return false;
  }
}

bool slab_supported(int n0, int n1, int n2) {
  if (n1 != n2 || !slab_plane(n1)) return false;
  switch (n0) {
#define X(n) case n:
    XFFT_FAST_SIZES(X)
#undef X
    return true;
    default:
      return false;
  }
}

size_t slab_table_floats(int n0, int n1) { return (size_t)slab::kGF * n0 * ((size_t)n1 * n1 / 2); }

int slab_z_blocks(int n0) { return 3 * n0; }

cudaError_t slab_green_table(float* table, int n0, int n1, const void* const* ge, const void* const* gs,
                             const double* ih, double halfvol, cudaStream_t s) {
  switch (n1) {
#define X(n) \
  case n:    \
    return slab::green_table_n<n>(table, n0, ge, gs, ih, halfvol, s);
    XFFT_SLAB_SMALL(X)
    X(128)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t slab_precondition(int n0, int n1, float* f, float* z, void* spec, long long stride, long long sstride,
                              const int* active, const void* tw0, const void* tw1, const void* tw2,
                              const float* table, const void* const* ge, const void* const* gs,
                              const double* ih, double halfvol, unsigned long long* units, const float* q,
                              const RhsState* st, double* partials, int nparts, int n_rhs, cudaStream_t s) {
  switch (n1) {
#define X(n)                                                                                                  \
  case n:                                                                                                     \
    return slab::precondition_n<n>(n0, f, z, spec, stride, sstride, active, tw0, tw1, tw2, table, ge, gs, ih, \
                                   halfvol, units, q, st, partials, nparts, n_rhs, s);
    XFFT_SLAB_SMALL(X)
    X(128)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace xfft
