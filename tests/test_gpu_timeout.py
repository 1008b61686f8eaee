"""Failure detection without a GPU fault: a bounded device wait on an mbarrier
that nothing arrives at gives up after its budget, the call reports
JET_ERR_TIMEOUT, and the context stays usable for the next call."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2606_29702_gb300 import jet, specs
    assert jet.debug_wait_timeout(2_000_000) == 6  # JET_ERR_TIMEOUT
    assert b"budget" in jet.load().jet_last_error()
    # the context still runs kernels
    plan = jet.Plan(specs.burgers(0.01), [2, 32, 32, 1], "bf16")
    p = torch.zeros(plan.info()["n_params"], device="cuda") + 0.1
    x = torch.rand(100, 2, device="cuda")
    r, loss = plan.forward(p, x)
    torch.cuda.synchronize()
    assert torch.isfinite(loss)
    assert jet.debug_wait_timeout(10) == 1  # out-of-range budget is rejected on the host
