"""torch.autograd.Function wrappers: the gradients autograd returns are the
hand-written adjoints of the CUDA library (render backward; adjoint trace),
checked against the direct C-ABI calls and against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_helpers import oracle_sensor
from test_gpu_trace_adjoint import config3_params, param_scales, perturbed

pytestmark = pytest.mark.gpu


def small_scene(seed=5, H=48, W_=40, ks=9):
    rng = np.random.default_rng(seed)
    aif = rng.random((2, 3, H, W_))
    depth = rng.uniform(0.4, 2.5, size=(2, H, W_))
    fh = np.array([0.0, 0.02, 0.05], dtype=np.float32)
    dm = np.array([0.5, 1.0, 2.0], dtype=np.float32)
    bank = rng.random((3, 3, 3, 2, ks, ks))
    bank /= bank.sum(axis=(3, 4, 5), keepdims=True)
    return aif, depth, bank, fh, dm


def test_render_autograd_matches_adjoint_and_oracle(sdlib):
    sd = sdlib
    aif, depth, bank, fh, dm = small_scene()
    ks = bank.shape[-1]
    lay = sd.BankLayout(fh, dm, 3, ks, 0.003)
    a = torch.tensor(aif, dtype=torch.float32, device="cuda", requires_grad=True)
    b = torch.tensor(bank.reshape(-1), dtype=torch.float32, device="cuda", requires_grad=True)
    d = torch.tensor(depth, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(11)
    go = rng.standard_normal((2, 6) + aif.shape[2:])
    gout = torch.tensor(go, dtype=torch.float32, device="cuda")
    out = sd.dp_render_autograd(a, b, d, lay)
    (out * gout).sum().backward()
    ga, gb = sd.dp_render_backward(gout, a.detach(), d, b.detach(), lay)
    torch.cuda.synchronize()
    # bank gradient: fixed-order sums, identical; image gradient: float
    # atomics in arbitrary order
    assert torch.equal(b.grad, gb)
    torch.testing.assert_close(a.grad, ga, rtol=1e-5, atol=1e-6)
    ref_a, ref_b = O.render_bank_bwd(go, aif.astype(np.float32).astype(np.float64),
                                     depth.astype(np.float32), bank.astype(np.float32)
                                     .astype(np.float64), fh, dm, 0.003)
    ea = np.abs(a.grad.cpu().numpy() - ref_a).max() / np.abs(ref_a).max()
    eb = np.abs(b.grad.cpu().numpy().reshape(ref_b.shape) - ref_b).max() / np.abs(ref_b).max()
    assert ea <= 1e-5 and eb <= 1e-5, (ea, eb)


def test_render_autograd_only_requested_gradients(sdlib):
    sd = sdlib
    aif, depth, bank, fh, dm = small_scene(seed=6)
    lay = sd.BankLayout(fh, dm, 3, bank.shape[-1], 0.003)
    a = torch.tensor(aif, dtype=torch.float32, device="cuda", requires_grad=True)
    b = torch.tensor(bank.reshape(-1), dtype=torch.float32, device="cuda")
    d = torch.tensor(depth, dtype=torch.float32, device="cuda")
    out = sd.dp_render_autograd(a, b, d, lay)
    out.square().sum().backward()
    assert a.grad is not None and b.grad is None
    assert torch.isfinite(a.grad).all()


def test_trace_autograd_matches_adjoint_and_descends(sdlib):
    """The trace as a differentiable function of the config-3 parameters:
    autograd's gradient is the adjoint trace's, and a small step against it
    lowers the config-3 loss sum (PSF - T)^2 as the first-order model
    predicts."""
    sd = sdlib
    cfg = W.config_full_forward()
    tab, ps, focus = cfg["lens"], cfg["pitch_mm"], cfg["focus_mm"]
    info = O.lens_info(tab, focus)
    reqs = W.bank_grid([0.0, 0.7, 1.3], [450.0, 1100.0], [W.LAMBDA_D, W.LAMBDA_F], 64, 65)
    S = oracle_sensor(ps)
    tgt, _ = O.psf_bank(perturbed(tab, info), 0.0, reqs, S, O.MODE_BILINEAR, O.NORM_PER_RAY,
                        n_threads=8)
    T = torch.tensor(np.concatenate([x.ravel() for x in tgt]), dtype=torch.float32,
                     device="cuda")
    pids = config3_params(tab)
    lens = sd.Lens(tab, focus)
    # nominal values of the parameters in set_param units (curvature 1/mm)
    theta0 = []
    for pid in pids:
        s, j = divmod(pid, 8)
        if j == 0:
            theta0.append(1.0 / tab[s, W.COL_R])
        elif j == 1:
            theta0.append(tab[s, W.COL_K])
        elif j == 7:
            theta0.append(info["sensor_dist"] if s == tab.shape[0] - 1 else tab[s, W.COL_T])
        else:
            theta0.append(tab[s, W.COL_A4 + j - 2])
    theta0 = np.array(theta0)
    dev, total, off = sd.make_requests(reqs)
    sen = sd.DPSensor(ps)

    def loss_at(th, grad=False):
        t = torch.tensor(th, dtype=torch.float64, requires_grad=grad)
        psf = sd.dp_psf_trace_autograd(t, lens, pids, sen, dev, len(reqs), total, max_ks=65,
                                       max_n=64)
        loss = (psf - T).square().sum()
        if grad:
            loss.backward()
            return loss.item(), t.grad.numpy().copy(), psf.detach()
        return loss.item()

    l0, g, psf0 = loss_at(theta0, grad=True)
    # the forward is the plain bilinear, per-ray normalised trace (its FP32
    # shared-memory splat adds in arbitrary order: equal to rounding)
    mask = sd.land_mask(len(reqs), 64)
    ref_psf, _ = sd.dp_psf_trace(lens, sen, dev, len(reqs), total, max_ks=65, max_n=64,
                                 mode=sd.SD_BIN_BILINEAR, norm=sd.SD_NORM_PER_RAY, mask=mask)
    torch.testing.assert_close(psf0, ref_psf, rtol=1e-5, atol=1e-9)
    # autograd's gradient is the adjoint trace of dLoss/dPSF = 2 (PSF - T),
    # restricted like autograd's to the rays the forward's landing mask marks
    _, glens = sd.dp_psf_trace_backward(lens, sen, dev, len(reqs), 2.0 * (psf0 - T), max_ks=65,
                                        max_n=64, mask=mask)
    direct = glens[0].reshape(-1).cpu().numpy()[pids].astype(np.float64)
    np.testing.assert_allclose(g, direct, rtol=1e-6, atol=1e-12 * np.abs(direct).max())
    # a step in natural units whose predicted decrease is 1 % of the loss
    h = param_scales(tab, info, pids)
    dirn = -(g * h) * h
    pred = float(-(g @ dirn))
    alpha = 0.01 * l0 / pred
    l1 = loss_at(theta0 + alpha * dirn)
    print(f"loss {l0:.6e} -> {l1:.6e}, predicted decrease {alpha * pred:.3e}")
    assert l0 - l1 >= 0.3 * alpha * pred
    lens.free()
