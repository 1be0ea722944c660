"""The allocation-free entry point biot_residual_norms_noalloc.

Callers that hand all GPU memory to their own pool cannot let the library call
cudaMalloc; for them the library offers one entry point whose scratch is a fixed
device array instead. This test gives it caller-owned device buffers (made here
with PyTorch, as such a caller's pool would) and checks, on two calls in a row,
that it returns what the context entry point biot_residual_norms returns for the
same state. The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


def _device_system(ctx, case):
    """Device copies of the arrays the entry point reads, derived from the ABI's exports."""
    rowptr, col, val, ap = biot.biot_get_csr(ctx)
    nn = case.n_nodes
    nodeptr = (rowptr[0:3 * nn + 1:3] // 9).astype(np.int32)   # rowptr[3v] = 9 * nodeptr[v]
    nodeptr[-1] = rowptr[-1] // 9
    nbr = np.empty(nodeptr[-1], dtype=np.int32)
    for v in range(nn):
        a = rowptr[3 * v]
        deg = nodeptr[v + 1] - nodeptr[v]
        nbr[nodeptr[v]:nodeptr[v + 1]] = col[a:a + 3 * deg:3] // 3
    diag = np.array([val[rowptr[r] + np.nonzero(col[rowptr[r]:rowptr[r + 1]] == r)[0][0]]
                     for r in range(3 * nn)])
    dsc = 1.0 / np.sqrt(np.abs(diag))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return {"nodeptr": dev(nodeptr), "nbr": dev(nbr), "rowptr": dev(rowptr), "val": dev(val), "ap": dev(ap),
            "dsc": dev(dsc)}, dsc


@pytest.mark.parametrize("name,lo", [("terzaghi", 1), ("mms_ragged", 3)])
def test_noalloc_matches_context_entry_point(name, lo):
    base = W.terzaghi_small()
    case = base if name == "terzaghi" else base.with_(n=9, problem="mms", E=2.0, kappa=0.5, tau=0.05, n_t=41)
    rng = np.random.default_rng(5)
    stream = torch.cuda.current_stream()
    with biot.Context(case, stream=stream) as c:
        X = rng.standard_normal((case.n_t + 1, case.n_dof)) * np.where(np.arange(case.n_dof) % 3 == 2, 1.0, 1e-4)
        biot.biot_set_state(c.ctx, 0, case.n_t, X)
        hi = case.n_t
        ncols = hi - lo + 1
        rel_ref = biot.biot_residual_norms(c.ctx, lo, hi)
        R_ref = biot.biot_get_residual(c.ctx, lo, hi)            # r (not equilibrated), [ncols][N_dof]
        F = biot.biot_get_rhs(c.ctx)
        sysd, dsc = _device_system(c.ctx, case)
    ldx = case.n_t + 1
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()       # [N_dof][ldx], time fastest
    Fd = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    ldr = ncols + 3
    for call in range(2):
        Rd = torch.full((case.n_dof, ldr), np.nan, dtype=torch.float64, device="cuda")
        reld = torch.full((ncols,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        biot.biot_residual_norms_noalloc(case.n_nodes, sysd["nodeptr"].data_ptr(), sysd["nbr"].data_ptr(),
                                         sysd["rowptr"].data_ptr(), sysd["val"].data_ptr(), sysd["ap"].data_ptr(),
                                         sysd["dsc"].data_ptr(), Xd.data_ptr(), Fd.data_ptr(), ldx, lo, ncols,
                                         Rd.data_ptr(), ldr, reld.data_ptr(), stream)
        torch.cuda.synchronize()
        if call == 1:
            # the defining property: a call after the first takes no device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        rel = reld.cpu().numpy()
        R = Rd.cpu().numpy()[:, :ncols].T / dsc                      # undo the equilibration
        np.testing.assert_allclose(rel, rel_ref, rtol=1e-12, atol=0)
        scale = np.abs(R_ref).max()
        assert np.abs(R - R_ref).max() <= 1e-13 * scale, call


def test_noalloc_rejects_oversized_window():
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = z.data_ptr()
    with pytest.raises(biot.BiotError) as e:
        biot.biot_residual_norms_noalloc(4, p, p, p, p, p, p, p, p, 600, 1, 513, p, 513, p)
    assert e.value.status == biot.BIOT_E_INVALID
    assert "1..512" in biot.biot_last_error(None)


def test_noalloc_rejects_window_past_int32():
    # lo + ncols beyond 2^31 - 1 must be rejected, not wrapped around
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = z.data_ptr()
    with pytest.raises(biot.BiotError) as e:
        biot.biot_residual_norms_noalloc(4, p, p, p, p, p, p, p, p, 100, 2**31 - 10, 20, p, 20, p)
    assert e.value.status == biot.BIOT_E_INVALID
