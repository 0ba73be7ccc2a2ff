"""The event loop computes the binary64 waiting time tau = E / (A 2^-32) and
the clock test t + tau < dt with integer instructions; they must equal the
IEEE round-to-nearest results of the GPU's FP64 unit bit for bit."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import tissue as T  # noqa: E402


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_time_path_matches_fp64_unit(seed):
    assert T.selftest_time(1 << 28, seed) == 0
