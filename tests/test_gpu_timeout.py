"""Failure detection without a GPU fault: a bounded wait that runs out.

The band triangular solves stage their band rows into shared memory by bulk copies and
wait for each block's copy with a bounded spin. When that wait runs out the kernel records
the failure in the context's device status, waits (with the full budget) for the copies
still in flight, and returns; biot_pint_solve then reports BIOT_E_TIMEOUT and the context
stays usable. The test shortens only that first wait (biot_debug_set_wait_budget) so that it
runs out, checks the status and message, restores the budget and checks that a fresh solve
on the same context converges to the oracle's sequential solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle.solvers import field_rel_errors, seq_solve
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


def test_wait_timeout_is_reported_and_context_recovers():
    # 16^2 mesh: plain band factors, the TMA-staged band solve (16-row blocks) by default
    case = W.terzaghi_small().with_(n_t=6)
    stream = torch.cuda.current_stream()
    ref = seq_solve(build_system(case))
    with biot.Context(case, stream=stream) as c:
        try:
            biot.biot_debug_set_wait_budget(1)
            with pytest.raises(biot.BiotError) as e:
                biot.biot_pint_solve(c.ctx, case.tol, 50)
            assert e.value.status == biot.BIOT_E_TIMEOUT
            assert "bounded device wait" in biot.biot_last_error(c.ctx)
        finally:
            biot.biot_debug_set_wait_budget(0)
        torch.cuda.synchronize()
        biot.biot_set_state(c.ctx, 1, case.n_t, np.zeros((case.n_t, case.n_dof)))
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 2000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    assert rel <= 1e-12
    eu, ep = field_rel_errors(X, ref)
    assert eu < 1e-10 and ep < 1e-10, (eu, ep)
