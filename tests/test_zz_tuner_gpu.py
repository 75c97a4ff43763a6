"""The autotuner on the GPU: it measures real design iterations, its choice is the fastest
admissible candidate, the solver built with the chosen options still meets the field
tolerance against the oracle, and a second call reads the cache."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fdfd_oracle as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2307_05388_gb300 import autograd as AG  # noqa: E402
from paper_2307_05388_gb300 import autotune as AT  # noqa: E402
from paper_2307_05388_gb300 import fdfd as FD  # noqa: E402
from tests import _gpu_util as U  # noqa: E402


def test_autotune_c1(tmp_path):
    wl = W.make("c1")
    eps_bg = torch.from_numpy(wl.eps_bg.reshape(-1).copy()).cuda()
    cols, g = U.monitor_tensors(wl)
    b = U.rhs_tensor(wl)

    def make(opts):
        s = FD.Solver(wl.nx, wl.ny, wl.dx, U.k0_of(wl), wl.npml, box=wl.box, options=opts)
        return AG.DesignProblem(s, eps_bg, b, cols, g)

    path = str(tmp_path / "tune.json")
    search = (("tensor_form", (3, 2)), ("tensor_min_m", (128, 1)))
    res = AT.tune(make, U.eps_design_tensor(wl, wl.rho), search=search, steps=2, warmup=1, cache_path=path)
    ok = [t for t in res.trials if t.ok]
    print("autotune c1:", [(t.params, t.ms, t.status) for t in res.trials])
    assert ok and res.params in [t.params for t in ok]
    assert min(t.ms for t in ok) == [t.ms for t in ok if t.params == res.params][0]
    assert all(t.ms is not None and t.ms > 0 for t in ok)

    # the chosen options meet the field tolerance, forward and transpose
    s = FD.Solver(wl.nx, wl.ny, wl.dx, U.k0_of(wl), wl.npml, box=wl.box, options=res.options)
    eps = wl.eps_full()
    s.factor(torch.from_numpy(eps.reshape(-1).copy()).cuda())
    rhs = W.random_complex((wl.n_omega, 1, wl.n), 11)
    fac = O.Factor(O.assemble(wl.nx, wl.ny, eps, wl.k0dx()[0], wl.npml))
    for tr in (False, True):
        x = s.solve(torch.from_numpy(rhs).cuda(), transpose=tr).cpu().numpy()
        ref = fac.solve_T(rhs[0, 0]) if tr else fac.solve(rhs[0, 0])
        assert O.rel_err(x.reshape(-1), ref) <= 1e-8
    s.close()

    again = AT.tune(make, U.eps_design_tensor(wl, wl.rho), search=search, cache_path=path, key=res.key)
    assert again.cached and again.params == res.params
    np.testing.assert_equal(AT.options_dict(again.options), AT.options_dict(res.options))
