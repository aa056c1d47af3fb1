"""Host-side checks of the Python binding (no GPU): the allocation-free entry
point sees only a raw device pointer, so its wrapper must refuse tensors of
the wrong dtype, shape, layout or device before anything is launched."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1412_3387_gb300 import md  # noqa: E402


@pytest.mark.parametrize("make,what", [
    (lambda: torch.zeros((8, 4), dtype=torch.float32), "float64"),
    (lambda: torch.zeros((8, 3), dtype=torch.float64), "shape"),
    (lambda: torch.zeros((8, 4, 1), dtype=torch.float64), "shape"),
    (lambda: torch.zeros((4, 8), dtype=torch.float64).t(), "contiguous"),
    (lambda: torch.zeros((8, 4), dtype=torch.float64), "CUDA"),
    (lambda: np.zeros((8, 4)), "torch tensor"),
])
def test_noalloc_wrapper_refuses_bad_tensors_before_launch(make, what):
    with pytest.raises(ValueError, match=what):
        md.lj_forces_noalloc(make(), [10.0, 10.0, 10.0], 2.5)
