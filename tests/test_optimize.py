"""The L-BFGS-B host loop on the CPU, with an objective whose optimum under the box bounds is
known in closed form (the GPU objective chain it drives is covered by the parity tests)."""
import numpy as np
import pytest
import torch

pytest.importorskip("scipy")
from paper_2307_05388_gb300 import optimize as OPT  # noqa: E402


def test_lbfgsb_maximises_under_the_box_bounds():
    """F = -sum (rho - c)^2 with c partly outside [0, 1]: the maximiser is clip(c, 0, 1)."""
    rng = np.random.default_rng(0)
    c = torch.from_numpy(rng.uniform(-0.5, 1.5, (6, 5)))
    calls = []

    def obj(rho):
        calls.append(rho.shape)
        return -((rho - c) ** 2).sum(), -2 * (rho - c)

    rho, F, res = OPT.lbfgsb(obj, torch.full((6, 5), 0.5, dtype=torch.float64), maxiter=50)
    assert rho.shape == (6, 5) and rho.dtype == torch.float64
    np.testing.assert_allclose(rho.numpy(), np.clip(c.numpy(), 0, 1), atol=1e-6)
    assert F == pytest.approx(-float(((np.clip(c.numpy(), 0, 1) - c.numpy()) ** 2).sum()), abs=1e-9)
    assert all(s == (6, 5) for s in calls)


def test_lbfgsb_minimise_and_callback():
    c = torch.linspace(0.1, 0.9, 8, dtype=torch.float64)
    seen = []
    rho, F, _ = OPT.lbfgsb(lambda r: (((r - c) ** 2).sum(), 2 * (r - c)), torch.zeros(8, dtype=torch.float64),
                           maximize=False, callback=lambda k, f, x: seen.append(f))
    np.testing.assert_allclose(rho.numpy(), c.numpy(), atol=1e-6)
    assert F == pytest.approx(0.0, abs=1e-10) and seen and seen[-1] <= seen[0]
