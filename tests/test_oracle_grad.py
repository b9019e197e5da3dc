"""FP64 gradient checks of the oracle's adjoint under a multi-resolution
log-magnitude loss (CPU, no GPU).

The adjoint of the real-signal analysis map (the adjoint of Algorithm 3:
Algorithm 4's steps with the analysis windows g_k and h_0) is the backward
of the forward transform.  Here torch's gradcheck compares it, in float64,
with central finite differences of the forward transform itself, under the
loss the differentiation workload uses:

    L(x) = sum_B mean_{m,n,k} | log(|c_B(x)| + eps) - log(|c_B(t)| + eps) |

over B = 12, 24, 48 bins per octave (fmin 40 Hz), t a fixed target signal.
Inputs: 4096 samples at 44.1 kHz, slice 2N = 1024, transition 256.
"""

import numpy as np
import pytest

import oracle as O
from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")

FS, N_SAMPLES, SLICE, TRANS, EPS = 44100.0, 4096, 1024, 256, 1e-6
RESOLUTIONS = (12, 24, 48)


def _plans():
    return [O.make_plan(O.SliCQParams(FS, 40.0, FS / 2, B, SLICE, TRANS)) for B in RESOLUTIONS]


class _OracleSliCQ(torch.autograd.Function):
    """Forward: the oracle's real-signal sliCQ; backward: the oracle's adjoint."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        ctx.n = x.shape[-1]
        return torch.from_numpy(O.slicq_forward(x.detach().numpy(), plan))

    @staticmethod
    def backward(ctx, grad_c):
        # torch hands the conjugate-Wirtinger gradient dL/dc-bar (times 2);
        # for real x the chain rule gives Re(A^H grad_c)
        g = O.slicq_adjoint(grad_c.detach().numpy(), ctx.plan, ctx.n)
        return torch.from_numpy(np.ascontiguousarray(g)), None


def _logmag_l1(c, ct):
    return (torch.log(c.abs() + EPS) - torch.log(ct.abs() + EPS)).abs().mean()


def _loss(x, targets, plans):
    return sum(_logmag_l1(_OracleSliCQ.apply(x, p), ct) for p, ct in zip(plans, targets))


def _inputs():
    noisy, clean = signals.noisy_clean_tone_mixtures(1, N_SAMPLES, FS, seed=signals.seed_for(4))
    return noisy[0].astype(np.float64), clean[0].astype(np.float64)


def test_adjoint_is_backward_gradcheck_fp64():
    """torch.autograd.gradcheck (FP64, finite differences of the oracle's
    forward) of the multi-resolution log-magnitude L1 loss."""
    plans = _plans()
    noisy, clean = _inputs()
    targets = [torch.from_numpy(O.slicq_forward(clean, p)) for p in plans]
    x = torch.from_numpy(noisy).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: _loss(v, targets, plans), (x,), eps=1e-7,
                                    atol=1e-6, rtol=1e-4, fast_mode=True)


def test_loss_directional_derivatives_fp64():
    """<grad L, v> from the adjoint equals a central difference of L along
    several random directions v (slow-mode check on a few directions)."""
    plans = _plans()
    noisy, clean = _inputs()
    targets = [torch.from_numpy(O.slicq_forward(clean, p)) for p in plans]
    x = torch.from_numpy(noisy).requires_grad_(True)
    loss = _loss(x, targets, plans)
    (g,) = torch.autograd.grad(loss, x)
    rng = np.random.default_rng(11)
    h = 1e-7
    for _ in range(3):
        v = torch.from_numpy(rng.standard_normal(N_SAMPLES))
        with torch.no_grad():
            fd = (_loss(x + h * v, targets, plans) - _loss(x - h * v, targets, plans)) / (2 * h)
        got = float(torch.dot(g, v))
        assert abs(got - float(fd)) <= 1e-5 * max(abs(float(fd)), 1e-3), (got, float(fd))


def test_zero_loss_at_target():
    """x = t gives L = 0 (every term vanishes), and a changed input a positive loss."""
    plans = _plans()
    _, clean = _inputs()
    targets = [torch.from_numpy(O.slicq_forward(clean, p)) for p in plans]
    assert float(_loss(torch.from_numpy(clean), targets, plans)) == 0.0
    assert float(_loss(torch.from_numpy(1.5 * clean), targets, plans)) > 0.0
