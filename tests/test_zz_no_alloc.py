"""GPU: qmc_slater_invert_noalloc, the re-inversion for callers that cannot allocate
device memory (their memory belongs to their own pool allocator, or they cannot afford
the synchronisation an allocation may bring), gives the results of the allocating
qmc_slater_invert, on two calls in a row with different inputs, and refuses a batch
larger than its fixed 16 MiB work area.

The file is named so that pytest collects it last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_06922_gb300 import qmcgb as q   # noqa: E402


def _inputs(seed, batch, n, dtype):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(batch, n, n)) + 2 * np.eye(n)
    return torch.tensor(A, dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_allocating_call_twice(dtype):
    for call, (batch, n) in enumerate([(5, 96), (3, 130)]):
        A = _inputs(100 + call, batch, n, dtype)
        B_ref = torch.empty_like(A)
        B_new = torch.full_like(A, float("nan"))
        ld_ref = torch.empty(batch, dtype=torch.float64, device="cuda")
        sg_ref = torch.empty_like(ld_ref)
        ld_new = torch.full_like(ld_ref, float("nan"))
        sg_new = torch.full_like(ld_ref, float("nan"))
        q.slater_invert(A, B_ref, ld_ref, sg_ref)
        q.slater_invert_noalloc(A, B_new, ld_new, sg_new)
        torch.cuda.synchronize()
        rtol = 1e-12 if dtype == torch.float64 else 1e-6
        scale = B_ref.abs().max()
        assert torch.all((B_new - B_ref).abs() <= rtol * scale), call
        assert torch.allclose(ld_new, ld_ref, rtol=1e-12, atol=0), call
        assert torch.equal(sg_new, sg_ref), call


def test_noalloc_refuses_a_batch_beyond_its_work_area():
    A = torch.zeros((33, 256, 256), dtype=torch.float64, device="cuda")   # 33 * 65536 > 2^21
    with pytest.raises(q.QMCError) as err:
        q.slater_invert_noalloc(A, A)
    assert err.value.status == q.QMC_EINVAL
    assert "work area" in str(err.value)


def test_noalloc_allocates_no_device_memory():
    """After a first call (which may make the runtime load the work area), further calls
    leave the device's free memory unchanged: nothing is allocated on their behalf."""
    batch, n = 4, 128
    A = _inputs(7, batch, n, torch.float64)
    B = torch.empty_like(A)
    ld = torch.empty(batch, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(ld)
    q.slater_invert_noalloc(A, B, ld, sg)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        q.slater_invert_noalloc(A, B, ld, sg)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
