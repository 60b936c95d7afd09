"""qst_adjoint_noalloc, the adjoint for callers that cannot call cudaMalloc
(code under an allocator it does not own, or loops that must not pay
cudaMalloc's implicit synchronisation): its workspace is a fixed device array
inside the library.  It must give the same adjoint as the plan-based
qst_adjoint, on repeated calls that reuse the shared scratch, and must refuse
problems larger than that scratch.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2607_19577_b300 import qst, synth

pytestmark = pytest.mark.gpu

G_TOL, H_TOL = 1e-4, 1e-4  # the tolerances of the parity tests


def _rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_noalloc_adjoint_matches_plan_adjoint_on_two_calls():
    inst = synth.random_instance(11, 60, 3, 800, 4242)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda()
    w = torch.from_numpy(inst.w).cuda()
    _, c_obs, _ = plan.forward(psi, w, data)
    g_ref, gw_ref = plan.adjoint(psi, w, data, c_obs)
    torch.cuda.synchronize()
    g_ref = g_ref.cpu().numpy()
    gw_ref = gw_ref.cpu().numpy()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        g = torch.full_like(psi, float("nan"))
        gw = torch.full_like(w, float("nan"))
        rc = qst.adjoint_noalloc(psi, w, data, c_obs, g, gw, status)
        assert rc == qst.QST_OK
        torch.cuda.synchronize()
        assert status.item() == 0
        g, gw = g.cpu().numpy(), gw.cpu().numpy()
        for k in range(inst.K):
            assert _rel_err(g[k], g_ref[k]) <= G_TOL
        np.testing.assert_allclose(gw, gw_ref, rtol=H_TOL)
    plan.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    inst = synth.random_instance(8, 6, 2, 100, 4343)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda()
    w = torch.from_numpy(inst.w).cuda()
    c_obs = torch.ones(inst.nnz, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # n = 16, K = 16 and 4096 settings need far more than the scratch; the call
    # must refuse before touching any pointer.
    big = qst.Data(n=16, basis=data.basis, row_ptr=data.row_ptr, outcome=data.outcome, count=data.count,
                   shots=data.shots)
    big_psi = torch.empty(16, 1 << 16, dtype=torch.complex64, device="cuda")
    object.__setattr__(big, "basis", torch.zeros(4096, 16, dtype=torch.uint8, device="cuda"))
    rc = qst.adjoint_noalloc(big_psi, torch.ones(16, device="cuda"), big, c_obs, big_psi, w, status)
    assert rc == qst.QST_ERR_SCRATCH_TOO_SMALL
