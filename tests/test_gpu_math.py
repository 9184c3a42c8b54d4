"""The trace's branch-free division and square root (reciprocal estimates
with one Newton-Raphson correction) against correctly rounded IEEE FP32
results: within one ulp over the operand ranges of the trace."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def ulp_dist(a, b):
    """Distance in units in the last place between FP32 arrays of equal sign."""
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def run(sd, a, b):
    from paper_2503_11213_gb300 import _lib as L
    from paper_2503_11213_gb300 import api
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
    q = torch.empty_like(ta)
    r = torch.empty_like(ta)
    L.check(L.lib().sd_dev_math_check(api._ptr(ta), api._ptr(tb), len(a), api._ptr(q),
                                      api._ptr(r), api._stream()), "sd_dev_math_check")
    torch.cuda.synchronize()
    return q.cpu().numpy(), r.cpu().numpy()


def test_division_and_sqrt_within_one_ulp(sdlib):
    rng = np.random.default_rng(0)
    n = 1 << 20
    a = (np.exp(rng.uniform(np.log(1e-6), np.log(1e6), n)) *
         rng.choice([-1.0, 1.0], n)).astype(np.float32)
    b = (np.exp(rng.uniform(np.log(1e-6), np.log(1e6), n)) *
         rng.choice([-1.0, 1.0], n)).astype(np.float32)
    q, r = run(sdlib, a, b)
    ref_q = a / b                       # float32 IEEE, correctly rounded
    assert np.all(np.sign(q) == np.sign(ref_q))
    dq = ulp_dist(q, ref_q)
    absa = np.abs(a)
    ref_r = np.sqrt(absa)
    _, r2 = run(sdlib, absa, b)
    dr = ulp_dist(r2, ref_r)
    print(f"div: max {dq.max()} ulp, {np.mean(dq > 0):.3%} not correctly rounded; "
          f"sqrt: max {dr.max()} ulp, {np.mean(dr > 0):.3%} not correctly rounded")
    assert dq.max() <= 1 and dr.max() <= 1
    # cosine-like operands near 1 and lengths of the trace
    c = rng.uniform(0.5, 1.0, n).astype(np.float32)
    _, rc = run(sdlib, c, c)
    assert ulp_dist(rc, np.sqrt(c)).max() <= 1


def test_sqrt_of_zero_is_tiny_not_nan(sdlib):
    q, r = run(sdlib, np.zeros(4, np.float32), np.ones(4, np.float32))
    assert np.all(q == 0) and np.all(np.isfinite(r)) and np.all(r <= 1e-14)
