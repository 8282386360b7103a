"""GPU adjoint: pfc_step_adjoint and the checkpointed autograd rollout against the FP64 oracle's
adjoint and against central finite differences.

Tolerances: FP64 adjoint step 1e-12 (relative L2 of lam, relative dr); rollout gradients vs the
oracle 1e-10; finite differences 1e-6 relative (FP64, the bar set for the adjoint). FP32-mixed
adjoint step 2e-5 (single-precision transforms around an O(1) multiplier range).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ONE = (0, -0.25, 0.0, 0.0)
TWO = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))


def _plan(shape, dt, op, prec):
    from paper_2603_26818_gb300 import binding
    return binding.Plan(shape, math.pi / 4, dt, [binding.make_op(*op)], precision=prec)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("shape,op,dt", [((64, 64), ONE, 0.5), ((16, 32, 32), TWO, 0.1),
                                         ((4096, 16), ONE, 0.5), ((512, 16, 16), TWO, 0.1)])
def test_adjoint_step_matches_oracle(shape, op, dt, prec, tol):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    psi = inputs.uniform_state(shape, -0.25, 0.2, seed=51)
    lam = inputs.uniform_state(shape, 0.0, 1.0, seed=52)
    ref_lam, ref_dr = oracle.step_adjoint(psi, lam, math.pi / 4, dt, op)
    p = _plan(shape, dt, op, prec)
    pd = torch.from_numpy(psi).to(device="cuda", dtype=dtype)
    ld = torch.from_numpy(lam).to(device="cuda", dtype=dtype)
    out = torch.empty_like(ld)
    dr = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")   # accumulates onto 0.5
    p.step_adjoint(pd, ld, out, dr)
    torch.cuda.synchronize()
    assert rel(out.double().cpu().numpy(), ref_lam) <= tol
    assert abs(float(dr) - 0.5 - ref_dr) <= tol * max(1.0, abs(ref_dr)) * 10
    # lam_out may alias lam_next
    p.step_adjoint(pd, ld, ld, dr)
    torch.cuda.synchronize()
    assert rel(ld.double().cpu().numpy(), ref_lam) <= tol


def _loss_and_grads(shape, dt, op, prec, nsteps, every, psi0, target, r):
    from paper_2603_26818_gb300.autograd import rollout
    dtype = torch.float64 if prec == "fp64" else torch.float32
    p = _plan(shape, dt, op, prec)
    x0 = torch.from_numpy(psi0).to(device="cuda", dtype=dtype).requires_grad_(True)
    rt = torch.tensor(r, dtype=torch.float64, requires_grad=True)
    tg = torch.from_numpy(target).to(device="cuda", dtype=dtype)
    out = rollout(x0, rt, p, nsteps, every)
    loss = 0.5 * ((out - tg) ** 2).sum()
    loss.backward()
    return float(loss.detach()), x0.grad.double().cpu().numpy(), float(rt.grad)


@pytest.mark.parametrize("shape,op,dt", [((32, 32), ONE, 0.5), ((16, 16, 32), TWO, 0.1)])
def test_rollout_gradients_match_oracle_adjoint(shape, op, dt):
    nsteps = 9
    psi0 = inputs.uniform_state(shape, -0.25, 0.1, seed=53)
    target = oracle.step(psi0, math.pi / 4, dt, (op[0], op[1] + 0.05, op[2], op[3]), nsteps)
    ref_loss, ref_g, ref_gr = oracle.adjoint_run(psi0, target, math.pi / 4, dt, op, nsteps)
    loss, g, gr = _loss_and_grads(shape, dt, op, "fp64", nsteps, 4, psi0, target, op[1])
    assert loss == pytest.approx(ref_loss, rel=1e-10)
    assert rel(g, ref_g) <= 1e-10
    assert gr == pytest.approx(ref_gr, rel=1e-10)


def test_checkpoint_interval_does_not_change_gradients():
    shape, dt, nsteps = (32, 32), 0.5, 12
    psi0 = inputs.uniform_state(shape, -0.25, 0.1, seed=54)
    target = inputs.uniform_state(shape, -0.25, 0.1, seed=55)
    a = _loss_and_grads(shape, dt, ONE, "fp64", nsteps, 1, psi0, target, -0.25)
    b = _loss_and_grads(shape, dt, ONE, "fp64", nsteps, 5, psi0, target, -0.25)
    c = _loss_and_grads(shape, dt, ONE, "fp64", nsteps, 12, psi0, target, -0.25)
    for x in (b, c):
        assert rel(x[1], a[1]) <= 1e-12
        assert x[2] == pytest.approx(a[2], rel=1e-12)


def test_adjoint_config_256_cubed_r_gradient_matches_finite_differences():
    """3D one-mode 256^3 FP64, dx = pi/4, dt = 0.5, r = -0.25, psi0 = -0.25 + U[-0.01, 0.01]
    (seed 6), 200 steps with checkpoints every 20; target = the same run at r = -0.2;
    loss = 0.5 ||psi_T - target||^2. dL/dr from the adjoint vs central differences in r."""
    from paper_2603_26818_gb300 import binding
    shape, dt, nsteps, every = (256, 256, 256), 0.5, 200, 20
    psi0 = inputs.uniform_state(shape, -0.25, 0.01, seed=6)
    p = _plan(shape, dt, ONE, "fp64")
    x0 = torch.from_numpy(psi0).cuda()

    def run(r):
        p.set_r(r)
        x = x0.clone()
        p.step(x, nsteps)
        return x

    tg = run(-0.2)
    loss, g, gr = _loss_and_grads(shape, dt, ONE, "fp64", nsteps, every, psi0, tg.cpu().numpy(), -0.25)
    # the loss varies like exp(-2 k^2 t r) over t = 100, so a second-order difference would carry
    # a truncation error of ~3e-6 at h = 2e-5: use the fourth-order central difference
    h = 2e-5
    L = lambda r: 0.5 * float(((run(r) - tg) ** 2).sum())
    fd = (8 * (L(-0.25 + h) - L(-0.25 - h)) - (L(-0.25 + 2 * h) - L(-0.25 - 2 * h))) / (12 * h)
    assert gr == pytest.approx(fd, rel=1e-6)
    assert np.isfinite(g).all()
    p.close()


@pytest.mark.parametrize("shape,op,dt", [((4096, 4096), ONE, 0.5), ((256, 256, 512), TWO, 0.1)])
def test_adjoint_step_on_the_clustered_row_passes(shape, op, dt):
    """FP32 adjoint step of plans whose psi^3 row pass runs on two-block clusters (2D rows of
    4096, 3D rows of 512) against the oracle's adjoint step."""
    psi = inputs.uniform_state(shape, -0.25, 0.2, seed=53)
    lam = inputs.uniform_state(shape, 0.0, 1.0, seed=54)
    ref_lam, ref_dr = oracle.step_adjoint(psi, lam, math.pi / 4, dt, op)
    p = _plan(shape, dt, op, "fp32")
    assert p.info()["row_cluster"] == 2
    pd = torch.from_numpy(psi).to(device="cuda", dtype=torch.float32)
    ld = torch.from_numpy(lam).to(device="cuda", dtype=torch.float32)
    out = torch.empty_like(ld)
    dr = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.step_adjoint(pd, ld, out, dr)
    torch.cuda.synchronize()
    assert rel(out.double().cpu().numpy(), ref_lam) <= 2e-5
    assert abs(float(dr) - ref_dr) <= 2e-4 * max(1.0, abs(ref_dr))
    p.close()


def test_adjoint_config_256_cubed_psi0_gradient_matches_finite_differences():
    """The same 256^3 FP64 workload: the initial-field gradient along a random direction v,
    <dL/dpsi0, v>, against the fourth-order central difference of L(psi0 + h v)."""
    shape, dt, nsteps, every = (256, 256, 256), 0.5, 200, 20
    psi0 = inputs.uniform_state(shape, -0.25, 0.01, seed=6)
    v = inputs.uniform_state(shape, 0.0, 1.0, seed=66)
    p = _plan(shape, dt, ONE, "fp64")
    p.set_r(-0.2)
    tg = torch.from_numpy(psi0).cuda()
    p.step(tg, nsteps)
    p.set_r(-0.25)
    loss, g, gr = _loss_and_grads(shape, dt, ONE, "fp64", nsteps, every, psi0, tg.cpu().numpy(), -0.25)
    gv = float(np.dot(g.ravel(), v.ravel()))
    x0 = torch.from_numpy(psi0).cuda()
    vd = torch.from_numpy(v).cuda()

    def L(h):
        x = x0 + h * vd
        p.step(x, nsteps)
        return 0.5 * float(((x - tg) ** 2).sum())

    h = 1e-5
    fd = (8 * (L(h) - L(-h)) - (L(2 * h) - L(-2 * h))) / (12 * h)
    print(f"256^3 FP64: <dL/dpsi0, v> adjoint {gv:.12e}, finite difference {fd:.12e}")
    assert gv == pytest.approx(fd, rel=1e-6)
    p.close()


def test_adjoint_config_256_cubed_fp32_gradients_against_fp64():
    """Config 5 in FP32-mixed: the rollout gradients (psi0 and r) against the FP64 ones on the
    same workload. The step is linearly unstable (r + 3 mean^2 < 0), so rounding differences of
    the FP32 forward run grow with the unstable modes over t = 100 before the adjoint carries
    them back; the bound is the relative L2 the arithmetic gives (FP32 transforms ~1e-7 per step,
    amplified along the unstable band), checked loosely and reported."""
    shape, dt, nsteps, every = (256, 256, 256), 0.5, 200, 20
    # one FP32-representable start and one target for both precisions
    psi0 = inputs.uniform_state(shape, -0.25, 0.01, seed=6).astype(np.float32).astype(np.float64)
    p = _plan(shape, dt, ONE, "fp64")
    p.set_r(-0.2)
    tg = torch.from_numpy(psi0).cuda()
    p.step(tg, nsteps)
    p.close()
    target = tg.float().double().cpu().numpy()
    res = {}
    for prec in ("fp64", "fp32"):
        res[prec] = _loss_and_grads(shape, dt, ONE, prec, nsteps, every, psi0, target, -0.25)
    (l64, g64, r64), (l32, g32, r32) = res["fp64"], res["fp32"]
    eg, er = rel(g32, g64), abs(r32 - r64) / abs(r64)
    print(f"256^3 adjoint FP32 vs FP64: loss {l32:.6e} / {l64:.6e}, rel L2 dL/dpsi0 {eg:.3e}, rel dL/dr {er:.3e}")
    assert np.isfinite(g32).all()
    assert eg <= 1e-3 and er <= 1e-3


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("shape,op,dt", [((64, 64), ONE, 0.5), ((16, 32, 32), TWO, 0.1), ((256, 128), ONE, 0.5),
                                         ((32, 32, 64), ONE, 0.5)])
def test_recorded_segment_adjoint_matches_step_by_step_adjoint(shape, op, dt, prec, tol):
    """pfc_step_record + pfc_adjoint_segment (lam kept in the internal layout, the fused adjoint
    row pass) against pfc_step applied step by step and pfc_step_adjoint applied in reverse."""
    dtype = torch.float64 if prec == "fp64" else torch.float32
    n = 7
    p = _plan(shape, dt, op, prec)
    nbytes = p.record_bytes(n)
    assert nbytes is not None
    psi0 = torch.from_numpy(inputs.uniform_state(shape, -0.25, 0.1, seed=57)).to(device="cuda", dtype=dtype)
    lam0 = torch.from_numpy(inputs.uniform_state(shape, 0.0, 1.0, seed=58)).to(device="cuda", dtype=dtype)
    # reference: the states step by step, the one-step adjoint in reverse
    traj = [psi0.clone()]
    for _ in range(n):
        z = traj[-1].clone()
        p.step(z, 1)
        traj.append(z)
    lam_ref = lam0.clone()
    dr_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in reversed(range(n)):
        p.step_adjoint(traj[k], lam_ref, lam_ref, dr_ref)
    # recorded segment
    rec = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    x = psi0.clone()
    p.step_record(x, n, rec)
    lam = lam0.clone()
    dr = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.adjoint_segment(rec, n, lam, dr)
    torch.cuda.synchronize()
    assert rel(x.double().cpu().numpy(), traj[-1].double().cpu().numpy()) <= (1e-14 if prec == "fp64" else 1e-6)
    assert rel(lam.double().cpu().numpy(), lam_ref.double().cpu().numpy()) <= tol
    assert float(dr) == pytest.approx(float(dr_ref), rel=tol * 10, abs=1e-12)
    p.close()


def test_segment_adjoint_is_unsupported_where_the_fused_row_pass_does_not_fit():
    """Two-field plans and FP32 rows of 4096 (two row buffers of a group exceed shared memory)
    report UNSUPPORTED, and the autograd rollout then falls back to the one-step adjoint."""
    from paper_2603_26818_gb300 import binding
    p = binding.Plan((32, 32), math.pi / 4, 0.5, [binding.make_op(*ONE), binding.make_op(*ONE)], precision="fp64",
                     coupling=0.1)
    assert p.record_bytes(4) is None
    p.close()
    q = _plan((4096, 4096), 0.5, ONE, "fp32")
    assert q.record_bytes(4) is None
    q.close()
