"""qst_adjoint_noalloc, the adjoint for callers that cannot call cudaMalloc
(code under an allocator it does not own, or loops that must not pay
cudaMalloc's implicit synchronisation): its workspace is a fixed device array
inside the library.  It must give the same adjoint as the plan-based
qst_adjoint (and as the FP64 oracle), on repeated calls that reuse the shared
scratch, including shapes with high qubits above the chunk and a capped bin
size, and must refuse problems larger than that scratch.  The binding rejects
malformed arguments before any pointer reaches the library.  This file is
collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth

G_TOL, H_TOL = 1e-4, 1e-4  # the tolerances of the parity tests


def _rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.gpu
@pytest.mark.parametrize("n,M,K,shots,seed,params", [
    (11, 60, 3, 800, 4242, None),                       # chunk = n: no high qubits
    (13, 40, 2, 600, 4244, None),                       # one high qubit: 3 bin keys
    (14, 40, 2, 600, 4245, None),                       # two high qubits: 9 bin keys
    (14, 40, 2, 600, 4246, {"max_bin_settings": 8}),    # capped bins: more bins, larger z buffer
])
def test_noalloc_adjoint_matches_plan_adjoint_on_two_calls(n, M, K, shots, seed, params):
    inst = synth.random_instance(n, M, K, shots, seed)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi = torch.from_numpy(inst.psi).cuda()
    w = torch.from_numpy(inst.w).cuda()
    _, c_obs, _ = plan.forward(psi, w, data)
    g_ref, gw_ref = plan.adjoint(psi, w, data, c_obs)
    torch.cuda.synchronize()
    g_ref = g_ref.cpu().numpy()
    gw_ref = gw_ref.cpu().numpy()
    ref = oracle.adjoint(n, inst.basis, inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                         inst.row_ptr, inst.outcome, c_obs.cpu().numpy().astype(np.float64))
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        g = torch.full_like(psi, float("nan"))
        gw = torch.full_like(w, float("nan"))
        rc = qst.adjoint_noalloc(psi, w, data, c_obs, g, gw, status, params=params)
        assert rc == qst.QST_OK
        torch.cuda.synchronize()
        assert status.item() == 0
        g, gw = g.cpu().numpy(), gw.cpu().numpy()
        for k in range(inst.K):
            assert _rel_err(g[k], g_ref[k]) <= G_TOL
            assert _rel_err(g[k], ref["grad_psi"][k]) <= G_TOL
        np.testing.assert_allclose(gw, gw_ref, rtol=H_TOL)
        np.testing.assert_allclose(gw, ref["grad_w"], rtol=H_TOL)
    plan.close()


@pytest.mark.gpu
def test_noalloc_rejects_problems_beyond_its_scratch():
    # n = 16, K = 16 and 4096 settings need far more than the scratch; the call
    # must refuse before touching any pointer.  No outcome is observed (nnz = 0),
    # so every argument is well-formed and cheap.
    n, M, K = 16, 4096, 16
    big = qst.Data(n=n, basis=torch.zeros(M, n, dtype=torch.uint8, device="cuda"),
                   row_ptr=torch.zeros(M + 1, dtype=torch.int64, device="cuda"),
                   outcome=torch.zeros(0, dtype=torch.int32, device="cuda"),
                   count=torch.zeros(0, dtype=torch.int32, device="cuda"),
                   shots=torch.ones(M, dtype=torch.int32, device="cuda"))
    psi = torch.zeros(K, 1 << n, dtype=torch.complex64, device="cuda")
    g = torch.empty_like(psi)
    w = torch.ones(K, device="cuda")
    gw = torch.empty_like(w)
    c_obs = torch.zeros(0, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = qst.adjoint_noalloc(psi, w, big, c_obs, g, gw, status)
    assert rc == qst.QST_ERR_SCRATCH_TOO_SMALL
    # the per-setting-round kernels only: another kernel family is refused
    small = synth.random_instance(8, 6, 2, 100, 4343)
    data = qst.Data.from_numpy(small.n, small.basis, small.row_ptr, small.outcome, small.count, small.shots)
    p2 = torch.from_numpy(small.psi).cuda()
    w2 = torch.from_numpy(small.w).cuda()
    rc = qst.adjoint_noalloc(p2, w2, data, torch.ones(small.nnz, device="cuda"), torch.empty_like(p2),
                             torch.empty_like(w2), status, params={"fixed_rounds": 2})
    assert rc == 1  # QST_ERR_INVALID_ARG


def test_noalloc_binding_rejects_bad_arguments_before_the_library(monkeypatch):
    """Malformed tensors raise QSTError in the binding; the library is never reached."""
    def no_library():
        raise AssertionError("the library must not be reached")
    monkeypatch.setattr(qst, "load", no_library)
    inst = synth.random_instance(6, 5, 2, 200, 4444)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots,
                               device="cpu")
    psi = torch.from_numpy(inst.psi)
    w = torch.from_numpy(inst.w)
    c = torch.ones(inst.nnz)
    st = torch.zeros(1, dtype=torch.int32)
    good = dict(psi=psi, w=w, d=data, c_obs=c, grad_psi=torch.empty_like(psi), grad_w=torch.empty_like(w),
                device_status=st)
    bad = {
        "power of two": dict(psi=torch.zeros(2, 48, dtype=torch.complex64)),
        "n = 7": dict(psi=torch.zeros(2, 128, dtype=torch.complex64), grad_psi=torch.zeros(2, 128, dtype=torch.complex64)),
        "grad_w": dict(grad_w=torch.empty(1)),
        "c_obs": dict(c_obs=torch.ones(inst.nnz - 1)),
        "grad_psi": dict(grad_psi=torch.empty(2, 64, dtype=torch.complex128)),
        "device_status": dict(device_status=torch.zeros(1, dtype=torch.int64)),
        "w:": dict(w=torch.ones(4)[::2]),
        "CUDA tensor": {},
    }
    for needle, change in bad.items():
        args = dict(good, **change)
        with pytest.raises(qst.QSTError) as e:
            qst.adjoint_noalloc(**args)
        assert needle in str(e.value), (needle, str(e.value))
