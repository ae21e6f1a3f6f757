"""Host-side argument checks of Solver.apply_noalloc (no GPU): every shape or placement
mismatch raises before anything reaches the library, which would otherwise read and write the
tensors through raw pointers sized by the row count and the DOF stride."""
import pytest

torch = pytest.importorskip("torch")

from paper_2601_02172_gb300.capi import check_noalloc_args  # noqa: E402

STRIDE = 30


def _t(*shape, dtype=None):
    return torch.zeros(shape, dtype=dtype or torch.float64)


@pytest.mark.parametrize("d,q,sig,exc", [
    (_t(2, STRIDE), _t(2, STRIDE), _t(2, 7), ValueError),          # host tensors: wrong device
    (_t(STRIDE), _t(STRIDE), None, ValueError),                    # 1-D d
    (_t(2, STRIDE + 1), _t(2, STRIDE + 1), None, ValueError),      # wrong row length
    (_t(2, STRIDE), _t(1, STRIDE), None, ValueError),              # short q
    (_t(2, STRIDE), _t(2, STRIDE), _t(2, 6), ValueError),          # short dAd_sig
    (_t(2, STRIDE), _t(2, STRIDE), _t(3, 7), ValueError),          # dAd_sig rows != k
    (_t(0, STRIDE), _t(0, STRIDE), None, ValueError),              # no rows
    (_t(2, STRIDE, dtype=torch.float32), _t(2, STRIDE, dtype=torch.float32), None, TypeError),
    (_t(2, STRIDE).numpy(), _t(2, STRIDE), None, TypeError),       # not a torch tensor
])
def test_mismatches_raise_before_any_launch(d, q, sig, exc):
    with pytest.raises(exc):
        check_noalloc_args(STRIDE, 0, d, q, sig)
