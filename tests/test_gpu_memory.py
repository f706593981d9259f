"""Plans' device memory comes from the library's pool: a plan freed and made
again reuses it (bit-identical results), and hmv_trim_memory hands the
unused part back to the device."""
import pytest

import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import uniform_vec

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


@pytest.mark.parametrize("method", [hmv.AUTO, hmv.NTT])
def test_plans_reuse_pooled_memory_and_trim_returns_it(method):
    torch = pytest.importorskip("torch")
    n, b = 700, 33220
    h = uniform_vec(31, 0, 2 * n - 1, b, 0)
    x = uniform_vec(31, 1, n, b, 0)
    want = None
    stream = torch.cuda.Stream()
    for _ in range(3):  # each plan reuses the memory the previous one freed
        with hmv.Plan(n, b, method=method, stream=stream.cuda_stream) as p:
            p.load_matrix(h)
            y = p.matvec(x)
        if want is None:
            want = y
        else:
            assert_same(y, want)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    hmv.trim_memory()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after - free_before >= hmv.plan_bytes(n, b, method=method) // 2
