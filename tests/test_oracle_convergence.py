"""Order of accuracy of the oracle on a curved mesh with a manufactured solution
(Sec. 6.1 regression practice: convergence rates from successive refinements).
Expected L2 order of the DGSEM solution: N+1."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, HLLC, Params

GAS = eq.Gas(1.4, 0.72, 1.0 / 1600.0)


def _error(N, nel, t_end, nt=0):
    m = wl.box_mesh((nel,) * 3, lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    dg = DGSEM(Params(N=N, node_type=nt, riemann=HLLC, mu=1.0 / 1600.0, bc_exact=eq.EXACT_MANUFACTURED, source=True),
               m.coords, m.conn)
    x = dg.geo.x.movedim(1, -1)
    U0 = eq.exact_state(eq.EXACT_MANUFACTURED, x, 0.0, GAS).movedim(-1, 1).contiguous()
    nsteps = int(math.ceil(t_end / (0.1 / nel / (N + 1))))
    dt = t_end / nsteps
    U = dg.run(U0, nsteps, dt)
    Ue = eq.exact_state(eq.EXACT_MANUFACTURED, x, t_end, GAS).movedim(-1, 1)
    wJ = dg.quad_weights()
    return math.sqrt(float((wJ * (U[:, 0] - Ue[:, 0]) ** 2).sum()))


@pytest.mark.parametrize("N", [2, 3])
def test_manufactured_solution_order(N):
    """Errors fall monotonically and the finest-pair order exceeds N.  At the
    resolutions a CPU test affords (2^3..8^3 elements over one wavelength) the
    observed orders are 2.35 (N=2) and 3.49 (N=3), i.e. pre-asymptotic between
    N and N+1; an inconsistent operator (dropped term, wrong sign) gives ~0."""
    errs = [_error(N, nel, 0.05) for nel in (2, 4, 8)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] > errs[1] > errs[2] and orders[-1] > N, (errs, orders)


def test_source_term_closed_form_inviscid_mass():
    """Mass equation of the manufactured field (u = 1 everywhere):
    S_rho = rho_t + div(rho u) = (-2 + 3) pi 0.1 cos(pi (x+y+z-2t))."""
    x = torch.tensor(np.random.default_rng(0).uniform(-1, 1, size=(7, 3)))
    S = eq.manufactured_source(x, 0.3, GAS)
    arg = math.pi * (x.sum(-1) - 0.6)
    assert torch.allclose(S[:, 0], 0.1 * math.pi * torch.cos(arg), rtol=1e-13, atol=1e-14)
