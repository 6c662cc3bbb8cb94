"""Differentiable unrolled A-MMMSE: the oracle's unrolled iteration, the
torch float64 reference gradient pinned to FP64 finite differences of the
oracle, and the CUDA forward pass and hand-written adjoint against both."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import model as om
from oracle import solvers as osv

from unrolled_ref import unrolled_wsr_torch


def _instance(shape, seed):
    rng = np.random.default_rng(seed)
    return wl.random_small(rng, *shape)


def _torch_args(inst):
    return (torch.from_numpy(inst.H[0].copy()), torch.from_numpy(inst.sigma2.copy()),
            torch.from_numpy(inst.alpha.copy()), float(inst.P[0]),
            torch.from_numpy(osv.initial_precoder(inst.G0, inst.P)[0].copy()))


def _oracle_wsr(inst, gammas, switch_iter):
    V0 = osv.initial_precoder(inst.G0, inst.P)
    return osv.ammmse_unrolled(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, gammas,
                               switch_iter)[1]


def _spectral_schedule(inst, T, switch_iter):
    """gamma_t = the spectral step 1/||F_k||_2 (eq. (16)) the solver takes at
    iteration t with the same stage schedule: the S5 value as initial steps."""
    V0 = osv.initial_precoder(inst.G0, inst.P)
    r = osv.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, T,
                   osv.Options(step_rule=1, switch_iter=switch_iter))
    return np.array([h.gamma[0] for h in r.history])


def _gammas(inst, T, scale=0.7):
    """Steps near the spectral value 1/||F||_2 at V^0 (W = I)."""
    V0 = osv.initial_precoder(inst.G0, inst.P)
    U = om.mmse_receiver(inst.H, V0, inst.sigma2, inst.K, inst.Nr, inst.d)
    g = om.spectral_step(inst.H, U, om.identity_weights(1, inst.K, inst.d), inst.alpha, 0, inst.K, inst.Nr)
    return np.array([scale * g * (1.0 + 0.05 * np.sin(t)) for t in range(T)])


SMALL = [((1, 3, 6, 2, 2), 11, 3), ((1, 2, 5, 3, 1), 12, -1), ((1, 4, 8, 2, 2), 13, 4)]


@pytest.mark.parametrize("shape,seed,sw", SMALL)
def test_torch_reference_matches_oracle(shape, seed, sw):
    inst = _instance(shape, seed)
    gam = _gammas(inst, 6)
    H, s2, al, P, V0 = _torch_args(inst)
    got = float(unrolled_wsr_torch(H, s2, al, P, V0, torch.from_numpy(gam), inst.K, inst.Nr, inst.d, sw))
    want = _oracle_wsr(inst, gam, sw)
    assert abs(got - want) <= 1e-10 * abs(want)


@pytest.mark.parametrize("shape,seed,sw", SMALL)
def test_torch_reference_gradient_matches_oracle_finite_differences(shape, seed, sw):
    """Autograd of the torch restatement against central FP64 differences
    of the oracle, for every gamma_t and for Re / Im of six entries of H."""
    inst = _instance(shape, seed)
    T = 6
    gam = _gammas(inst, T)
    H, s2, al, P, V0 = _torch_args(inst)
    Ht = H.clone().requires_grad_(True)
    gt = torch.from_numpy(gam).requires_grad_(True)
    unrolled_wsr_torch(Ht, s2, al, P, V0, gt, inst.K, inst.Nr, inst.d, sw).backward()
    for t in range(T):
        h = 1e-6 * gam[t]
        gp, gm = gam.copy(), gam.copy()
        gp[t] += h
        gm[t] -= h
        fd = (_oracle_wsr(inst, gp, sw) - _oracle_wsr(inst, gm, sw)) / (2 * h)
        assert abs(float(gt.grad[t]) - fd) <= 1e-5 * max(1.0, abs(fd)), (t, float(gt.grad[t]), fd)
    rng = np.random.default_rng(seed)
    for _ in range(6):
        i, q = rng.integers(inst.H.shape[1]), rng.integers(inst.H.shape[2])
        for part, unit in (("re", 1.0), ("im", 1j)):
            h = 1e-6
            Hp, Hm = inst.H.copy(), inst.H.copy()
            Hp[0, i, q] += unit * h
            Hm[0, i, q] -= unit * h
            ip, im_ = wl.Instance(**{**inst.__dict__, "H": Hp}), wl.Instance(**{**inst.__dict__, "H": Hm})
            fd = (_oracle_wsr(ip, gam, sw) - _oracle_wsr(im_, gam, sw)) / (2 * h)
            g = Ht.grad[i, q]
            got = float(g.real if part == "re" else g.imag)
            assert abs(got - fd) <= 1e-5 * max(1.0, abs(fd)), (part, i, q, got, fd)


# ---------------------------------------------------------------- GPU
def _gpu_run(insts, gam, T, ck, sw, want_grad=True):
    import paper_2510_20507_gb300 as pkg
    from gpu_util import to_dev
    from paper_2510_20507_gb300.unrolled import unrolled_wsr
    shape = (1, insts[0].K, insts[0].Nt, insts[0].Nr, insts[0].d)
    H = to_dev(np.stack([i.H[0] for i in insts]).astype(np.complex64))
    al = to_dev(np.stack([i.alpha for i in insts]).astype(np.float32))
    s2 = to_dev(np.stack([i.sigma2 for i in insts]).astype(np.float32))
    P = to_dev(np.array([i.P[0] for i in insts], dtype=np.float32))
    V0 = to_dev(np.stack([osv.initial_precoder(i.G0, i.P)[0] for i in insts]).astype(np.complex64))
    g = to_dev(np.asarray(gam, dtype=np.float32))
    solver = pkg.UnrolledSolver(len(insts), shape, T, ckpt_every=ck, switch_iter=sw)
    H.requires_grad_(want_grad)
    g.requires_grad_(want_grad)
    wsr = unrolled_wsr(solver, H, g, al, s2, P, V0)
    out = {"wsr": wsr.detach().cpu().numpy()}
    if want_grad:
        gb = torch.empty(len(insts), T, dtype=torch.float32, device="cuda:0")
        Hb = torch.empty_like(H)
        solver.backward(torch.ones(len(insts), dtype=torch.float64, device="cuda:0"), gb, Hb)
        st = solver.status(torch.empty(len(insts), dtype=torch.int32, device="cuda:0"))
        torch.cuda.synchronize()
        out.update(gamma_bar=gb.cpu().numpy().astype(np.float64), H_bar=Hb.cpu().numpy().astype(np.complex128),
                   status=st.cpu().numpy())
    solver.close()
    return out


def _rounded(insts):
    from gpu_util import round_inputs
    return round_inputs(insts)


@pytest.mark.gpu
@pytest.mark.parametrize("shape,seed,sw", SMALL)
def test_gpu_unrolled_matches_oracle_and_reference(shape, seed, sw):
    """Forward WSR against the oracle; per-instance gradients in every
    gamma_t and in H against the torch float64 reference (T = 8,
    checkpoints every 3 iterations, so segments are ragged)."""
    import __graft_entry__ as ge
    ge.build()
    T, ck = 8, 3
    insts = _rounded([_instance(shape, seed + 100 * b) for b in range(4)])
    gam = _gammas(insts[0], T).astype(np.float32).astype(np.float64)
    out = _gpu_run(insts, gam, T, ck, sw)
    assert np.all(out["status"] == 0)
    for b, inst in enumerate(insts):
        want = _oracle_wsr(inst, gam, sw)
        assert abs(out["wsr"][b] - want) <= 1e-5 * abs(want), (b, out["wsr"][b], want)
        H, s2, al, P, V0 = _torch_args(inst)
        Ht = H.clone().requires_grad_(True)
        gt = torch.from_numpy(gam).requires_grad_(True)
        unrolled_wsr_torch(Ht, s2, al, P, V0, gt, inst.K, inst.Nr, inst.d, sw).backward()
        rg = gt.grad.numpy()
        eg = np.linalg.norm(out["gamma_bar"][b] - rg) / np.linalg.norm(rg)
        rh = Ht.grad.numpy()
        eh = np.linalg.norm(out["H_bar"][b] - rh) / np.linalg.norm(rh)
        print(f"{shape} instance {b}: gamma grad rel err {eg:.2e}, H grad rel err {eh:.2e}")
        assert eg <= 1e-3 and eh <= 1e-3


@pytest.mark.gpu
def test_gpu_unrolled_gamma_gradient_against_oracle_finite_differences():
    """dWSR/dgamma_t from the CUDA adjoint against central FP64 differences
    of the oracle's unrolled iteration."""
    import __graft_entry__ as ge
    ge.build()
    T, ck, sw = 6, 2, 3
    inst = _rounded([_instance((1, 3, 6, 2, 2), 21)])[0]
    gam = _gammas(inst, T).astype(np.float32).astype(np.float64)
    out = _gpu_run([inst], gam, T, ck, sw)
    for t in range(T):
        h = 1e-6 * gam[t]
        gp, gm = gam.copy(), gam.copy()
        gp[t] += h
        gm[t] -= h
        fd = (_oracle_wsr(inst, gp, sw) - _oracle_wsr(inst, gm, sw)) / (2 * h)
        assert abs(out["gamma_bar"][0][t] - fd) <= 1e-3 * abs(fd) + 1e-6, (t, out["gamma_bar"][0][t], fd)


@pytest.mark.gpu
def test_gpu_unrolled_config_nt64_k16_t20():
    """Nt=64, K=16, Nr=2, d=2, P=20 dB, T=20, checkpoints every 5 (the
    unrolled workload): forward against the oracle on every instance of a
    batch of 8, gradients against the torch reference on two of them, and
    the autograd Function's gamma gradient as the sum over the batch."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg
    from gpu_util import to_dev
    from paper_2510_20507_gb300.unrolled import unrolled_wsr
    T, ck, sw = 20, 5, 4
    insts = _rounded(wl.unrolled_64(n=8))
    gam = _spectral_schedule(insts[0], T, sw).astype(np.float32).astype(np.float64)
    out = _gpu_run(insts, gam, T, ck, sw)
    assert np.all(out["status"] == 0)
    gaps = [abs(out["wsr"][b] - _oracle_wsr(inst, gam, sw)) / _oracle_wsr(inst, gam, sw)
            for b, inst in enumerate(insts)]
    print(f"unrolled Nt=64 K=16: WSR {np.round(out['wsr'], 3)}, max gap to the oracle {max(gaps):.2e}")
    assert max(gaps) <= 1e-4
    for b in (0, 5):
        inst = insts[b]
        H, s2, al, P, V0 = _torch_args(inst)
        Ht = H.clone().requires_grad_(True)
        gt = torch.from_numpy(gam).requires_grad_(True)
        unrolled_wsr_torch(Ht, s2, al, P, V0, gt, inst.K, inst.Nr, inst.d, sw).backward()
        eg = np.linalg.norm(out["gamma_bar"][b] - gt.grad.numpy()) / np.linalg.norm(gt.grad.numpy())
        eh = np.linalg.norm(out["H_bar"][b] - Ht.grad.numpy()) / np.linalg.norm(Ht.grad.numpy())
        print(f"unrolled Nt=64 K=16: instance {b}: gamma grad rel err {eg:.2e}, H grad rel err {eh:.2e}")
        assert eg <= 2e-3 and eh <= 2e-3
    # through torch.autograd: the batch's summed WSR
    H = to_dev(np.stack([i.H[0] for i in insts]).astype(np.complex64)).requires_grad_(True)
    g = to_dev(gam.astype(np.float32)).requires_grad_(True)
    al = to_dev(np.stack([i.alpha for i in insts]).astype(np.float32))
    s2 = to_dev(np.stack([i.sigma2 for i in insts]).astype(np.float32))
    P = to_dev(np.array([i.P[0] for i in insts], dtype=np.float32))
    V0 = to_dev(np.stack([osv.initial_precoder(i.G0, i.P)[0] for i in insts]).astype(np.complex64))
    solver = pkg.UnrolledSolver(len(insts), (1, 16, 64, 2, 2), T, ckpt_every=ck, switch_iter=sw)
    unrolled_wsr(solver, H, g, al, s2, P, V0).sum().backward()
    torch.cuda.synchronize()
    assert np.allclose(g.grad.cpu().numpy(), out["gamma_bar"].sum(0), rtol=1e-5, atol=1e-6)
    assert np.allclose(H.grad.cpu().numpy(), out["H_bar"], rtol=1e-5, atol=1e-6)
    solver.close()


@pytest.mark.gpu
def test_gpu_unrolled_two_forwards_then_backward():
    """Two graphs on one solver (e.g. two losses, or a validation pass in
    between): the backward of the first, taken after the second forward,
    gives the gradients of a lone forward/backward of the first; an in-place
    edit of H after a forward is refused by torch's version check."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg
    from gpu_util import to_dev
    from paper_2510_20507_gb300.unrolled import unrolled_wsr
    T, ck, sw = 6, 3, 3
    insts = _rounded([_instance((1, 3, 6, 2, 2), 900 + b) for b in range(4)])
    gam = _gammas(insts[0], T).astype(np.float32)

    def args(scale):
        H = to_dev((scale * np.stack([i.H[0] for i in insts])).astype(np.complex64)).requires_grad_(True)
        al = to_dev(np.stack([i.alpha for i in insts]).astype(np.float32))
        s2 = to_dev(np.stack([i.sigma2 for i in insts]).astype(np.float32))
        P = to_dev(np.array([i.P[0] for i in insts], dtype=np.float32))
        V0 = to_dev(np.stack([osv.initial_precoder(i.G0, i.P)[0] for i in insts]).astype(np.complex64))
        g = to_dev(gam.copy()).requires_grad_(True)
        return H, g, al, s2, P, V0

    solver = pkg.UnrolledSolver(len(insts), (1, 3, 6, 2, 2), T, ckpt_every=ck, switch_iter=sw)
    a = args(1.0)
    unrolled_wsr(solver, a[0], a[1], *a[2:]).sum().backward()
    want_H, want_g = a[0].grad.clone(), a[1].grad.clone()
    b, c = args(1.0), args(1.3)
    lb = unrolled_wsr(solver, b[0], b[1], *b[2:]).sum()
    lc = unrolled_wsr(solver, c[0], c[1], *c[2:]).sum()   # a second forward on the same solver
    lb.backward()
    assert torch.equal(b[0].grad, want_H) and torch.equal(b[1].grad, want_g)
    lc.backward()
    assert not torch.equal(c[0].grad, want_H)
    d = args(1.0)
    ld = unrolled_wsr(solver, d[0], d[1], *d[2:]).sum()
    with torch.no_grad():
        d[0].mul_(2.0)
    with pytest.raises(RuntimeError):
        ld.backward()
    solver.close()
