"""GPU discrete adjoint against the oracle's taped reverse sweep and finite differences.

* one adjoint step equals torch autograd's vector-Jacobian product of one
  oracle step (canonical state and Brinkman field), FP64, 1e-12;
* the checkpointed gradient of J(s) after T steps equals the taped FP64
  reverse of the oracle (1e-10 relative), for several checkpoint intervals;
* central differences of the GPU's own FP64 forward agree to 1e-6;
* FP32 storage + FP32 adjoint with FP64 accumulation stays within a stated
  bound of the FP64 gradient.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import adjoint as oadj
from oracle import lbm as olbm
from oracle import tables as otables
import paper_1410_0412_gb300 as lbm

pytestmark = pytest.mark.gpu


def _setup(seed=0, shape=(10, 9, 8), per=(1, 0, 1), xp=False, g=(1e-3, 0, 0)):
    solid = geometry.random_voxels(*shape, 0.15, 300 + seed)
    T = otables.Tables(solid, periodic=per, x_pressure=xp)
    lat = lbm.Lattice(solid, periodic=per, x_pressure=xp).upload()
    kw = dict(omega_plus=1.0, magic=3 / 16, g=g, rho_in=1.002 if xp else 1.0, rho_out=0.998 if xp else 1.0)
    op, lp = olbm.Params(**kw), lbm.Params(**kw)
    s = torch.as_tensor(geometry.uniform_field(T.N, 40 + seed), dtype=torch.float32) * 0.3
    return T, lat, op, lp, s


@pytest.mark.parametrize("ria", [False, True])
@pytest.mark.parametrize("xp", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f64df"])
def test_one_step_vjp(ria, xp, prec):
    T, lat, op, lp, s = _setup(1, per=(0, 0, 1) if xp else (1, 0, 1), xp=xp)
    gen = torch.Generator().manual_seed(3)
    F = olbm.uniform_state(T.N, op, 1.0, (0.02, -0.01, 0.0))
    F = F * (1 + 1e-2 * (torch.rand(F.shape, generator=gen, dtype=torch.float64) - 0.5))
    lam1 = torch.rand((19, T.N), generator=gen, dtype=torch.float64) - 0.5
    s64 = s.to(torch.float64)
    Fr = F.clone().requires_grad_(True)
    sr = s64.clone().requires_grad_(True)
    out = olbm.stream(olbm.collide(Fr, op, sr), T.adj, op)
    ref_lam, ref_gs = torch.autograd.grad(out, [Fr, sr], lam1)
    G = lat.new_grid(prec)
    lbm.lbm_load_canonical(lat, prec, lp, F.cuda(), G, lbm.LBM_LAYOUT_OSNT)
    ln = lbm.new_adjoint(lat, prec)
    ln[:, :T.N] = lam1.cuda()
    lo = lbm.new_adjoint(lat, prec)
    gs = torch.zeros(T.N, dtype=torch.float64, device="cuda")
    lbm.lbm_adjoint_step(lat, prec, lp, G, ln, lo, s.cuda(), gs, ria)
    got = lo[:, :T.N].cpu()
    assert float((got - ref_lam).abs().max() / ref_lam.abs().max()) <= 1e-12
    assert float((gs.cpu() - ref_gs).abs().max() / ref_gs.abs().max()) <= 1e-12


@pytest.mark.parametrize("K", [1, 3, 7, 20])
def test_checkpointed_gradient_vs_taped_oracle(K):
    T, lat, op, lp, s = _setup(2)
    steps = 20
    G0o = olbm.from_canonical(olbm.uniform_state(T.N, op), 0, T.adj, op)
    J_ref, dJ_ref, dF_ref = oadj.flux_and_gradient(G0o, T.adj, op, s.to(torch.float64), steps, wrt_state=True)
    G0 = lat.new_grid("f64")
    lbm.lbm_init_equilibrium(lat, "f64", lp, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
    ws = torch.empty((lbm.lbm_ckpt_workspace_bytes(lat, "f64", steps, K) + 7) // 8, dtype=torch.float64,
                     device="cuda")
    J = lbm.lbm_flux_forward(lat, "f64", lp, G0, s.cuda(), steps, K, ws, ria=True)
    lam0 = lbm.new_adjoint(lat, "f64")
    grad = lbm.lbm_flux_backward(lat, "f64", lp, s.cuda(), steps, K, ws, ria=True, lambda_0=lam0)
    assert abs(float(J) - float(J_ref)) <= 1e-13 * abs(float(J_ref))
    assert float((grad.cpu() - dJ_ref).abs().max() / dJ_ref.abs().max()) <= 1e-10
    # dJ/dG0 of the oracle is w.r.t. the OS-NT grid; lambda_0 is w.r.t. the canonical F_0 = stream(G0):
    # dJ/dG0 = S^T lambda_0
    lam = lam0[:, :T.N].cpu().clone().requires_grad_(False)
    Gv = G0o.clone().requires_grad_(True)
    (st,) = torch.autograd.grad(olbm.stream(Gv, T.adj, op), Gv, lam)
    assert float((st - dF_ref).abs().max() / dF_ref.abs().max()) <= 1e-10


def test_autograd_function_and_finite_differences():
    """dJ/ds from the adjoint vs central differences of the GPU FP64 forward (h = 1e-4)."""
    T, lat, op, lp, s = _setup(3, shape=(12, 10, 9), g=(1e-4, 0, 0))
    lp_shift = lbm.Params(omega_plus=lp.omega_plus, magic=lp.magic, g=lp.g, shifted=True)
    steps, K = 60, 8
    G0 = lat.new_grid("f64")
    lbm.lbm_init_equilibrium(lat, "f64", lp_shift, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
    sv = s.cuda().requires_grad_(True)
    J = lbm.flux_objective(sv, lat, "f64", lp_shift, G0, steps, K, ria=True)
    J.backward()
    g_auto = sv.grad.to(torch.float64)
    ws = torch.empty((lbm.lbm_ckpt_workspace_bytes(lat, "f64", steps, K) + 7) // 8, dtype=torch.float64,
                     device="cuda")
    lbm.lbm_flux_forward(lat, "f64", lp_shift, G0, s.cuda(), steps, K, ws, ria=True)
    g_adj = lbm.lbm_flux_backward(lat, "f64", lp_shift, s.cuda(), steps, K, ws, ria=True)
    assert torch.allclose(g_auto, g_adj.to(torch.float32).to(torch.float64), rtol=0, atol=0)
    h = 1e-4
    rng = np.random.default_rng(4)
    for n in rng.choice(T.N, 5, replace=False):
        vals = []
        for sign in (1, -1):
            sp = s.clone().to(torch.float64)
            sp[n] += sign * h
            # s is float32 in the library: keep the perturbed node exactly representable
            spf = sp.to(torch.float32)
            hh = float(spf[n].double() - s[n].double())
            Jv = lbm.lbm_flux_forward(lat, "f64", lp_shift, G0, spf.cuda(), steps, K, ws, ria=True)
            vals.append((float(Jv), hh))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        assert abs(fd - float(g_adj[n])) <= 1e-6 * abs(float(g_adj[n])) + 1e-16


def test_fp32_adjoint_error_vs_fp64():
    T, lat, op, lp, s = _setup(4, shape=(12, 10, 9), g=(1e-4, 0, 0))
    steps, K = 30, 6
    lps = lbm.Params(omega_plus=lp.omega_plus, magic=lp.magic, g=lp.g, shifted=True)
    grads = {}
    for prec in ("f64", "f32"):
        G0 = lat.new_grid(prec)
        lbm.lbm_init_equilibrium(lat, prec, lps, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
        ws = torch.empty((lbm.lbm_ckpt_workspace_bytes(lat, prec, steps, K) + 7) // 8, dtype=torch.float64,
                         device="cuda")
        lbm.lbm_flux_forward(lat, prec, lps, G0, s.cuda(), steps, K, ws, ria=False)
        grads[prec] = lbm.lbm_flux_backward(lat, prec, lps, s.cuda(), steps, K, ws, ria=False).cpu()
    rel = float((grads["f32"] - grads["f64"]).abs().max() / grads["f64"].abs().max())
    assert rel <= 1e-3


def test_config4_crop_vs_taped_oracle():
    """32^3 fully periodic crop of the Brinkman-field box (smoothed noise, sigma 3, seed 2),
    g = 1e-5 x, T = 100 steps, checkpoint every 10: FP64 gradient vs the taped oracle to 1e-10,
    FP32 storage with FP64 accumulation within the stated 1e-3."""
    n, steps, K = 32, 100, 10
    solid = geometry.empty_box(n, n, n)
    T = otables.Tables(solid, periodic=(1, 1, 1))
    lat = lbm.Lattice(solid, periodic=(1, 1, 1)).upload()
    field = geometry.smooth_noise(n, n, n, 3.0, 2)
    s = torch.as_tensor(geometry.node_field(field, T.node_xyz))
    kw = dict(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0.0, 0.0))
    op = olbm.Params(**kw)
    G0o = olbm.from_canonical(olbm.uniform_state(T.N, op), 0, T.adj, op)
    J_ref, dJ_ref = oadj.flux_and_gradient(G0o, T.adj, op, s.to(torch.float64), steps)
    for prec, tol in (("f64", 1e-10), ("f64df", 1e-10), ("f32", 1e-3)):
        lp = lbm.Params(shifted=(prec != "f64"), **kw)
        G0 = lat.new_grid(prec)
        lbm.lbm_init_equilibrium(lat, prec, lp, G0, lbm.LBM_LAYOUT_OSNT, 1.0)
        ws = torch.empty((lbm.lbm_ckpt_workspace_bytes(lat, prec, steps, K) + 7) // 8, dtype=torch.float64,
                         device="cuda")
        J = lbm.lbm_flux_forward(lat, prec, lp, G0, s.cuda(), steps, K, ws, ria=True)
        grad = lbm.lbm_flux_backward(lat, prec, lp, s.cuda(), steps, K, ws, ria=True).cpu()
        assert abs(float(J) - float(J_ref)) <= max(tol, 1e-13) * abs(float(J_ref))
        assert float((grad - dJ_ref).abs().max() / dJ_ref.abs().max()) <= tol
