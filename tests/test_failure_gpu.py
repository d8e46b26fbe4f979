"""Failure detection on the GPU without a fault: a bounded wait on a flag
that nothing sets gives up, the host reads ADPAR_ERR_TIMEOUT from the
workspace, and the same context and workspace then serve a normal call."""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(oracle):
    from paper_2202_10297_gb300 import adpar as A
    A.lib()
    work = A.workspace(1 << 20)
    A.adpar_selftest_timeout(work)
    assert A.adpar_workspace_status(work) == A.ERR_TIMEOUT
    # the context is still usable, and the workspace is reusable
    x = synth.normal(50001, np.float32, seed=1)
    y = synth.normal(50001, np.float32, seed=2)
    ab, _, _ = A.adpar_vjp_scan("max", torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), work=work)
    assert A.adpar_workspace_status(work) == A.OK
    ref, _, _, _ = oracle.scan_vjp("max", x, y)
    got = ab.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
