"""GPU: the standalone FP64 re-inversion (qmc_slater_invert) against LAPACK's LU
inverse and log-determinant, including ragged sizes and an exactly singular matrix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_06922_gb300 import qmcgb as q   # noqa: E402


@pytest.mark.parametrize("n", [1, 7, 8, 9, 70, 257, 520])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_invert_matches_lapack(n, dtype):
    rng = np.random.default_rng(n)
    batch = 3
    A = rng.normal(size=(batch, n, n)) + 2 * np.eye(n)
    Ad = torch.tensor(A, dtype=dtype, device="cuda")
    A_used = Ad.double().cpu().numpy()          # the values the kernel actually sees
    B = torch.empty_like(Ad)
    ld = torch.empty(batch, dtype=torch.float64, device="cuda")
    sg = torch.empty(batch, dtype=torch.float64, device="cuda")
    q.slater_invert(Ad, B, ld, sg)
    torch.cuda.synchronize()
    for b in range(batch):
        s_ref, l_ref = np.linalg.slogdet(A_used[b])
        ref = np.linalg.inv(A_used[b]).T
        got = B[b].double().cpu().numpy()
        tol = 1e-11 * np.linalg.cond(A_used[b]) if dtype == torch.float64 else 2.0 ** -23
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max() + 1e-300
        assert abs(ld[b].item() - l_ref) < 1e-11 * max(1.0, abs(l_ref))
        assert sg[b].item() == s_ref


def test_singular_matrix_is_reported():
    A = np.random.default_rng(0).normal(size=(2, 5, 5))
    A[1, :, 2] = 0.0            # an orbital that vanishes at every electron: a zero column
    Ad = torch.tensor(A, device="cuda")
    B = torch.full_like(Ad, 7.0)
    ld = torch.zeros(2, dtype=torch.float64, device="cuda")
    sg = torch.zeros(2, dtype=torch.float64, device="cuda")
    q.slater_invert(Ad, B, ld, sg)
    torch.cuda.synchronize()
    assert sg[1].item() == 0.0 and ld[1].item() == -np.inf
    assert torch.all(B[1] == 0)
    assert sg[0].item() != 0.0


def test_invert_rejects_bad_arguments():
    A = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        q.slater_invert(A.cpu(), A)                      # host memory, caught by the binding
    h = A.cpu()
    lib = q.load()                                       # and by the library itself
    assert lib.qmc_slater_invert(0, h.data_ptr(), A.data_ptr(), None, None, 4, 1, None) == q.QMC_EINVAL
    big = torch.zeros((1, 1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QMCError):
        q.slater_invert(big, big)


def test_invert_refuses_mismatched_buffers():
    """Shapes, dtypes and lengths are checked before the library is called (a short or
    mistyped buffer would otherwise be written past its end)."""
    A = torch.eye(8, dtype=torch.float64, device="cuda").expand(3, 8, 8).contiguous()
    bad = [
        (A, torch.empty(3, 8, 8, dtype=torch.float32, device="cuda"), None, None),   # dtype
        (A, torch.empty(2, 8, 8, dtype=torch.float64, device="cuda"), None, None),   # shape
        (A, torch.empty_like(A), torch.empty(2, dtype=torch.float64, device="cuda"), None),
        (A, torch.empty_like(A), None, torch.empty(3, dtype=torch.float32, device="cuda")),
        (A[:, :, :7].contiguous(), torch.empty(3, 8, 7, dtype=torch.float64, device="cuda"), None, None),
    ]
    for args in bad:
        for fn in (q.slater_invert, q.slater_invert_noalloc):
            with pytest.raises(ValueError):
                fn(*args)
