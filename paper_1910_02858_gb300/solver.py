"""User-facing wrapper: a Solver owns one library context; torch provides the
device memory and the stream.  All arithmetic runs in the CUDA kernels behind
include/flexi.h.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import flexi as F


@dataclass
class SolverConfig:
    N: int = 3
    Ngeo: int = 1
    node_type: int = F.NODES_GAUSS
    riemann: int = F.RIEMANN_ROE
    precision: int = F.FP64
    bc_exact: int = F.EXACT_TGV
    source: bool = False
    split_form: int = F.SPLIT_STANDARD
    adjoint: bool = False  # allocate the discrete adjoint's scratch
    lifting: int = F.LIFTING_BR1
    eta_br2: float = 2.0
    gamma: float = 1.4
    Pr: float = 0.72
    mu: float = 1.0 / 1600.0
    Ma: float = 0.1

    def to_c(self) -> F.flexi_params:
        return F.flexi_params(N=self.N, Ngeo=self.Ngeo, node_type=self.node_type, riemann=self.riemann,
                              precision=self.precision, bc_exact=self.bc_exact, source=int(self.source),
                              split_form=self.split_form, gamma=self.gamma, Pr=self.Pr, mu=self.mu, Ma=self.Ma,
                              adjoint=int(self.adjoint), lifting=self.lifting, eta_br2=self.eta_br2)


class Solver:
    def __init__(self, cfg: SolverConfig, coords: np.ndarray, conn: np.ndarray, device="cuda:0", mortars=None):
        self.cfg = cfg
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device)
            if mortars is not None and len(mortars) > 0:
                self.ctx = F.flexi_mesh_init_mortar(cfg.to_c(), coords, conn, mortars, stream)
            else:
                self.ctx = F.flexi_mesh_init(cfg.to_c(), coords, conn, stream)
        self.K = F.flexi_query(self.ctx, F.Q_K)
        self.n = cfg.N + 1
        self.dtype = torch.float64 if cfg.precision == F.FP64 else torch.float32

    # --------------------------------------------------------------
    def _stream(self):
        return torch.cuda.current_stream(self.device)

    def _check(self, *ts):
        for t in ts:
            if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
                raise ValueError(f"expected contiguous {self.dtype} tensors on {self.device}")
            if t.numel() != self.K * 5 * self.n ** 3:
                raise ValueError("wrong number of elements")

    def empty_state(self):
        return torch.empty(self.K, 5, self.n, self.n, self.n, dtype=self.dtype, device=self.device)

    def rhs(self, U, t=0.0, out=None):
        out = torch.empty_like(U) if out is None else out
        self._check(U, out)
        F.flexi_rhs(self.ctx, U, out, t, self._stream())
        return out

    def step(self, U, dU, t, dt):
        self._check(U, dU)
        F.flexi_rk_step(self.ctx, U, dU, t, dt, self._stream())

    def step_stages(self, U, dU, t, dt, stages):
        self._check(U, dU)
        F.flexi_rk_step_stages(self.ctx, U, dU, t, dt, stages, self._stream())

    def run(self, U, nsteps, dt, t0=0.0, graph=True):
        """Advance U (device tensor) in place by nsteps LSERK4(5) steps
        (flexi_rk_run: CUDA-graph replay of one step when the operator does not
        depend on t; graph=False launches every step)."""
        self._check(U)
        dU = getattr(self, "_dU", None)
        if dU is None or dU.shape != U.shape or dU.dtype != U.dtype:
            dU = self._dU = torch.zeros_like(U)
        dU.zero_()  # finite: A_1 = 0 multiplies it in the first stage
        if graph:
            F.flexi_rk_run(self.ctx, U, dU, nsteps, t0, dt, self._stream())
        else:
            for s in range(nsteps):
                self.step(U, dU, t0 + s * dt, dt)
        return U

    def rhs_adjoint(self, U, lam, t=0.0, out=None):
        out = torch.empty_like(U) if out is None else out
        self._check(U, lam, out)
        F.flexi_rhs_adjoint(self.ctx, U, lam, out, t, self._stream())
        return out

    def adjoint_step(self, stages, lamU, lam_dU, t, dt):
        self._check(lamU, lam_dU)
        F.flexi_adjoint_step(self.ctx, stages, lamU, lam_dU, t, dt, self._stream())

    def reduce(self, U, Ut=None, cfl=0.9, allow_nonphysical=False):
        vals, code = F.flexi_reduce(self.ctx, U, Ut, cfl, self._stream(), allow_nonphysical)
        keys = ["mass", "mom_x", "mom_y", "mom_z", "energy", "kinetic_energy", "dkedt", "dt_max"]
        out = dict(zip(keys, vals))
        out["status"] = code
        return out

    def set_bc(self, bc_id: int, kind: int):
        """Boundary kind (flexi.BC_*) of the sides with boundary id bc_id."""
        F.flexi_set_bc(self.ctx, bc_id, kind)

    def query(self, what):
        return F.flexi_query(self.ctx, what)

    def close(self):
        if getattr(self, "ctx", None):
            F.flexi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
