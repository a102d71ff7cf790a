"""Degenerate meshes and calls on the CUDA path, against the FP64 oracle.

- A single periodic element: every face of the element is its own neighbour's face
  (each side pairs two local sides of the same element).
- A mesh one element thick in one direction (periodic): the element is its own
  neighbour along that direction, its other faces are ordinary sides.
- Small N with several elements per CTA (N = 1: 8 elements, N = 2: 3 elements per
  CTA) and an element count that leaves the last CTA partly empty.
- The small-mesh lifting/volume kernels at n = 4 (FP64): a cluster of two CTAs per
  element when there are at most half as many elements as SMs (48 elements, Gauss and
  Gauss-Lobatto, reoriented sides), three thread groups in one CTA per element below
  one element per SM (100 elements).
- Zero steps: flexi_rk_run and flexi_rk_run_host leave the state unchanged.

Right-hand sides use the rounding-sensitivity tolerance of test_gpu_parity, states
after time steps 1e-12 relative L2 per conserved variable.
"""
import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _oracle, _solver, per_var_rel, rhs_parity_ok

pytestmark = pytest.mark.gpu

CASES = [
    # (name, mesh kwargs, solver kwargs)
    ("single_element_lg_N3_hllc", dict(nelem=(1, 1, 1)), dict(N=3, riemann=1)),
    ("single_element_lgl_N4_roe", dict(nelem=(1, 1, 1), reorient_seed=2), dict(N=4, node_type=1, riemann=0)),
    ("one_thick_lg_N4_hllc", dict(nelem=(1, 2, 3), reorient_seed=5), dict(N=4, riemann=1)),
    ("ragged_cta_lg_N1_roe", dict(nelem=(3, 1, 3), reorient_seed=3), dict(N=1, riemann=0)),  # 9 elements, 8 per CTA
    ("ragged_cta_lg_N2_hllc", dict(nelem=(2, 2, 2), reorient_seed=4), dict(N=2, riemann=1)),  # 8 elements, 3 per CTA
    ("cluster_pair_lg_N3_hllc", dict(nelem=(4, 4, 3), reorient_seed=6), dict(N=3, riemann=1)),
    ("cluster_pair_lgl_N3_roe", dict(nelem=(3, 4, 4), reorient_seed=8), dict(N=3, node_type=1, riemann=0)),
    ("three_groups_lg_N3_hllc", dict(nelem=(5, 5, 4), reorient_seed=7), dict(N=3, riemann=1)),
]


@pytest.mark.parametrize("name,mk,sk", CASES, ids=[c[0] for c in CASES])
def test_degenerate_mesh_rhs_and_steps(name, mk, sk):
    mesh = wl.box_mesh(Ngeo=1, **mk)
    sk = dict(sk, precision=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    N, nt = sk["N"], sk.get("node_type", 0)
    U0 = wl.perturbed(mesh.node_coords(N, nt), seed=17)
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.0)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.0, mesh)
    assert ok, (d, tol)
    U = torch.tensor(U0, device=DEV)
    s.run(U, 5, 2e-3)
    ref = dg.run(torch.tensor(U0), 5, 2e-3)
    s.close()
    err = per_var_rel(U, ref)
    assert err < 1e-12, err


def test_zero_steps_leave_the_state_unchanged():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2), Ngeo=1)
    s = _solver(dict(N=3, riemann=1), mesh)
    U0 = torch.tensor(wl.taylor_green(mesh.node_coords(3, 0)))
    Ud = U0.to(DEV)
    dU = torch.zeros_like(Ud)
    F.flexi_rk_run(s.ctx, Ud, dU, 0, 0.0, 1e-3, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.equal(Ud.cpu(), U0)
    Uh = U0.clone().pin_memory()
    F.flexi_rk_run_host(s.ctx, Uh, 0, 0.0, 1e-3, torch.cuda.current_stream())
    assert torch.equal(Uh, U0)
    s.close()
