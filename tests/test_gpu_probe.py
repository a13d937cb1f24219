"""The tensor-instruction peak probes (cup_probe_tensor_peak) that justify the tensor
engine's choice of instruction: each returns a positive rate, and the bounded wait of
the tcgen05 probe completes."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_probe_rates_are_positive(cuda_lib, kind):
    r = cuda_lib.probe_tensor_peak(kind, iters=200 if kind == 2 else 100)
    assert math.isfinite(r) and r > 0.0


def test_probe_rejects_bad_kinds(cuda_lib):
    with pytest.raises(cuda_lib.CupError):
        cuda_lib.probe_tensor_peak(3)
