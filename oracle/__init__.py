"""Oracle: a plain, slow, FP64 CPU implementation of the DGSEM right-hand side,
the low-storage Runge-Kutta step and its adjoint, written from the paper
(Krais et al., FLEXI, Sec. 3.1 and Sec. 3.4; Eqs. semiDiscrete, discreteGradient).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with the
CUDA path: the only common dependency is ``workloads`` (seeded input
generators, which hold none of the method's arithmetic).

Every step is a direct transcription of the cited equation in torch float64 CPU
ops, vectorised over elements/sides only; no blocking, fusion or reordering
beyond what the equations state.  Library primitives used as steps: tensor
contractions (torch.einsum / tensordot), and torch.autograd for the
vector-Jacobian products of the adjoint (exact reverse-mode derivative of this
very oracle).
"""
