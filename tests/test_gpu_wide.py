"""States of 17..20 qubits against the FP64 oracle: the default wide path
(chunk of n - 8 qubits, 8 high bits by butterfly passes, settings in groups)
and the cluster path (chunk_qubits = 16: 16-qubit chunks on 8-CTA clusters,
settings binned by the n - 16 high bits); and the n = 20, M = 1024, K = 8
workload on sampled outputs and identities."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_19577_b300 import qst, synth
from test_gpu_parity import compare, run_gpu, run_gpu_evaluate, run_oracle

pytestmark = pytest.mark.gpu


# (17, 40, 2, 3000): ~1500 outcomes per (setting, high pattern), past the 512 staged per setting
@pytest.mark.parametrize("n,M,K,shots,seed", [(17, 6, 2, 3000, 1), (17, 40, 2, 3000, 4), (18, 4, 2, 4000, 2),
                                              (19, 5, 3, 2000, 5), (20, 3, 2, 10000, 3)])
def test_cluster_parity(n, M, K, shots, seed):
    inst = synth.random_instance(n, M, K, shots, 500 + seed)
    compare(inst, run_gpu(inst, chunk_qubits=16), run_oracle(inst))


def test_cluster_dense_p_and_many_bins():
    """Dense p from round C's registers; 30 settings at n = 17 fill the three
    high-pattern bins, two of them split by max_bin_settings = 4."""
    inst = synth.random_instance(17, 30, 1, 800, 31)
    gpu = run_gpu(inst, dense=True, max_bin_settings=4, chunk_qubits=16)
    compare(inst, gpu, run_oracle(inst, dense=True), dense=True)


@pytest.mark.parametrize("n,M,K,shots,seed", [(17, 9, 3, 2000, 8), (20, 5, 2, 10000, 9)])
def test_cluster_evaluate_equals_forward_adjoint(n, M, K, shots, seed):
    """qst_evaluate reuses the forward's transforms; qst_adjoint recomputes them
    with the same forward kernel: both are bitwise equal, and match the oracle."""
    inst = synth.random_instance(n, M, K, shots, 700 + seed)
    ev = run_gpu_evaluate(inst, chunk_qubits=16)
    compare(inst, ev, run_oracle(inst))
    sep = run_gpu(inst, chunk_qubits=16)
    for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
        assert np.array_equal(ev[key], sep[key]), key
    assert ev["loss"] == sep["loss"]
    off = run_gpu_evaluate(inst, phi_cache=0, chunk_qubits=16)
    for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
        assert np.array_equal(ev[key], off[key]), key


def test_cluster_geometry_and_refusals():
    plan = qst.Plan(20, 8, 2, 100, chunk_qubits=16)
    assert plan.geometry() == {"chunk_qubits": 16, "high_qubits": 4, "fixed_rounds": 4}
    plan.close()
    plan = qst.Plan(20, 8, 2, 100)
    assert plan.geometry()["chunk_qubits"] == 12 and plan.geometry()["high_qubits"] == 8
    plan.close()
    plan = qst.Plan(17, 8, 2, 100, fixed_rounds=4)  # fixed_rounds = 4 asks for the cluster kernels
    assert plan.geometry() == {"chunk_qubits": 16, "high_qubits": 1, "fixed_rounds": 4}
    plan.close()
    with pytest.raises(qst.QSTError):
        qst.Plan(20, 8, 2, 100, chunk_qubits=16, fixed_rounds=2)  # the cluster kernels are the 16-qubit chunks' only kernels
    with pytest.raises(qst.QSTError):
        qst.Plan(16, 8, 2, 100, fixed_rounds=4)  # and run only 16-qubit chunks


@pytest.mark.parametrize("n,M,K,shots,seed", [(17, 6, 2, 3000, 1), (18, 4, 2, 4000, 2), (20, 3, 2, 10000, 3)])
def test_wide_parity(n, M, K, shots, seed):
    inst = synth.random_instance(n, M, K, shots, 500 + seed)
    compare(inst, run_gpu(inst, chunk_qubits=n - 8), run_oracle(inst))


def test_wide_parity_several_groups():
    """n = 17 puts 64 settings in a group; 70 settings need two groups."""
    inst = synth.random_instance(17, 70, 1, 500, 77)
    compare(inst, run_gpu(inst, chunk_qubits=9), run_oracle(inst))


@pytest.fixture(scope="module")
def c5():
    inst = synth.make_instance("n20_m1024_k8", seed=0)
    plan = qst.Plan(inst.n, inst.M, inst.K, inst.nnz)
    data = qst.Data.from_numpy(inst.n, inst.basis, inst.row_ptr, inst.outcome, inst.count, inst.shots)
    psi, w = torch.from_numpy(inst.psi).cuda(), torch.from_numpy(inst.w).cuda()
    p_obs, c_obs, loss = plan.forward(psi, w, data)
    g, gw = plan.adjoint(psi, w, data, c_obs)
    torch.cuda.synchronize()
    assert plan.status() == 0
    yield dict(inst=inst, plan=plan, data=data, psi=psi, w=w, p_obs=p_obs, c_obs=c_obs, loss=loss, g=g, gw=gw)
    plan.close()


def _rows(inst, sel):
    rp, outs, cnts = [0], [], []
    for s in sel:
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        outs.append(inst.outcome[lo:hi])
        cnts.append(inst.count[lo:hi])
        rp.append(rp[-1] + hi - lo)
    return np.array(rp, np.int64), np.concatenate(outs), np.concatenate(cnts)


def test_n20_sampled_forward(c5):
    inst = c5["inst"]
    sel = synth.rng_for(2024).choice(inst.M, 3, replace=False)
    rp, out, cnt = _rows(inst, sel)
    ref = oracle.forward(inst.n, inst.basis[sel], inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                         rp, out, cnt, inst.shots[sel], eps=inst.eps, B=inst.M)
    p = c5["p_obs"].cpu().numpy()
    c = c5["c_obs"].cpu().numpy()
    for j, s in enumerate(sel):
        lo, hi = inst.row_ptr[s], inst.row_ptr[s + 1]
        r = ref["p_obs"][rp[j]:rp[j + 1]]
        assert np.max(np.abs(p[lo:hi] - r)) / np.max(r) <= 1e-5
        np.testing.assert_allclose(c[lo:hi], ref["c_obs"][rp[j]:rp[j + 1]], rtol=1e-4)


def test_n20_sampled_adjoint(c5):
    inst = c5["inst"]
    sel = np.sort(synth.rng_for(7).choice(inst.M, 2, replace=False))
    mask = np.zeros(inst.nnz, bool)
    for s in sel:
        mask[inst.row_ptr[s]:inst.row_ptr[s + 1]] = True
    c_full = c5["c_obs"].cpu().numpy()
    g, gw = c5["plan"].adjoint(c5["psi"], c5["w"], c5["data"],
                               torch.from_numpy(np.where(mask, c_full, 0).astype(np.float32)).cuda())
    rp, out, _ = _rows(inst, sel)
    ref = oracle.adjoint(inst.n, inst.basis[sel], inst.psi.astype(np.complex128), inst.w.astype(np.float64),
                         rp, out, c_full[mask].astype(np.float64), B=inst.M)
    g = g.cpu().numpy().astype(np.complex128)
    for k in range(inst.K):
        assert np.max(np.abs(g[k] - ref["grad_psi"][k])) / np.max(np.abs(ref["grad_psi"][k])) <= 1e-4
    np.testing.assert_allclose(gw.cpu().numpy(), ref["grad_w"], rtol=1e-4)


def test_n20_identities(c5):
    inst = c5["inst"]
    psi = c5["psi"].cpu().numpy().astype(np.complex128)
    w = c5["w"].cpu().numpy().astype(np.float64)
    g = c5["g"].cpu().numpy().astype(np.complex128)
    h = -c5["gw"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(np.sum(np.conj(psi) * (-g / w[:, None]), axis=1).real, h, rtol=1e-4)
    c = c5["c_obs"].cpu().numpy().astype(np.float64)
    p = c5["p_obs"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(np.dot(w, h), np.sum(c * p / inst.M), rtol=1e-5)


@pytest.mark.parametrize("n,M,K,shots,seed", [(20, 3, 2, 10000, 12), (20, 7, 3, 3000, 13)])
def test_wide_evaluate_with_transform_cache(n, M, K, shots, seed):
    """The wide path with the transform cache (phi_cache = 1): qst_evaluate's
    adjoint skips the group's high pass and the forward rounds; against the oracle,
    and bitwise equal to qst_forward + qst_adjoint (which recompute).  Wide plans
    of n = 17..19 (chunks below 12 qubits) refuse the cache."""
    inst = synth.random_instance(n, M, K, shots, 600 + seed)
    ev = run_gpu_evaluate(inst, phi_cache=1, chunk_qubits=n - 8)
    compare(inst, ev, run_oracle(inst))
    sep = run_gpu(inst, phi_cache=1, chunk_qubits=n - 8)
    for key in ["p_obs", "c_obs", "grad_psi", "grad_w"]:
        assert np.array_equal(ev[key], sep[key]), key
    assert ev["loss"] == sep["loss"]
    with pytest.raises(qst.QSTError):
        qst.Plan(17, 4, 2, 10, phi_cache=1, chunk_qubits=9)
