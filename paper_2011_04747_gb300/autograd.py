"""torch.autograd wrapper of the discrete adjoint (libdaeti's daeti_adjoint).

``MonodomainMisfit.apply(d_node, tau_close, problem)`` returns the sensor
misfit L = sum_j sum_s (v_s(t_j) - d_js)^2 of a Mitchell-Schaeffer tissue on
a structured grid whose element conductivity is the mean of its nodal values,
and back-propagates dL/d(d_node) and dL/d(tau_close).  The library computes the
loss and both gradients in one call (forward with binomial checkpoints, then
the reverse sweep); its nodal entry points form the element means and apply
their chain rule to the gradient, so this wrapper only moves arrays.

The problem keeps one prepared solver: later calls replace its conductivity
(daeti_update_conductivity_nodal) and tau_close (daeti_update_cell_params)
and keep the prepared schedule (dt, l, k_max) and the adjoint's device
buffers; only an update that the prepared l cannot take stably
(DAETI_EUNSTABLE) prepares a new solver.  ``problem.close()`` frees it.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import binding


@dataclasses.dataclass
class MisfitProblem:
    dim: int
    n: tuple
    h: float
    ms_params: tuple            # tau_in, tau_out, tau_open, tau_close (replaced), v_gate
    stimuli: list               # objects with nodes, t_start, duration, amplitude, period, count
    sensors: np.ndarray
    data: np.ndarray            # (n_samples, n_sensors)
    n_steps: int
    sample_every: int = 10
    n_slots: int = 32
    precision: str = "fp32_kahan"
    dt: float = 0.1
    _solver: object = dataclasses.field(default=None, repr=False, compare=False)
    prepares: int = dataclasses.field(default=0, compare=False)   # solvers prepared so far

    def close(self):
        if self._solver is not None:
            self._solver.close()
            self._solver = None

    def elements(self):
        nx, ny = self.n[0], self.n[1]
        nz = self.n[2] if self.dim == 3 else 1
        ez_n = nz - 1 if self.dim == 3 else 1
        ez, ey, ex = np.meshgrid(np.arange(ez_n), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
        base = (ex + nx * (ey + ny * ez)).ravel()
        offs = [(a & 1) + nx * ((a >> 1) & 1) + nx * ny * ((a >> 2) & 1) for a in range(2 ** self.dim)]
        return base[:, None] + np.array(offs)[None, :]


def _prepare(problem: MisfitProblem, d_node: np.ndarray, params):
    s = binding.Solver(precision=problem.precision, dt=problem.dt, graph_steps=0)
    try:
        s.daeti_set_mesh_grid(problem.dim, problem.n, problem.h)
        s.daeti_set_conductivity_nodal(d_node)       # element D = mean of its nodes
        s.daeti_set_cell_model("ms", tuple(params))
        for st in problem.stimuli:
            s.daeti_add_stimulus(st.nodes, st.t_start, st.duration, st.amplitude, st.period, st.count)
        s.daeti_prepare()
    except Exception:
        s.close()
        raise
    problem.prepares += 1
    return s


def _solve(problem: MisfitProblem, d_node: np.ndarray, tau_close: float):
    params = list(problem.ms_params)
    params[3] = float(tau_close)
    s = problem._solver
    if s is not None:
        try:
            s.daeti_update_conductivity_nodal(d_node)
            s.daeti_update_cell_params(params)
        except binding.DaetiError as e:
            if e.code != binding.EUNSTABLE:
                raise
            problem.close()
            s = None
    if s is None:
        s = problem._solver = _prepare(problem, d_node, params)
    return s.daeti_adjoint(problem.sensors, problem.data, problem.n_steps, problem.sample_every,
                           problem.n_slots, 0, nodal=True)


class MonodomainMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d_node: torch.Tensor, tau_close: torch.Tensor, problem: MisfitProblem):
        loss, g_node, g_tau = _solve(problem, d_node.detach().cpu().double().numpy(), float(tau_close))
        ctx.save_for_backward(torch.as_tensor(g_node, dtype=d_node.dtype, device=d_node.device),
                              torch.as_tensor(g_tau, dtype=tau_close.dtype, device=tau_close.device))
        return torch.as_tensor(loss, dtype=torch.float64, device=d_node.device)

    @staticmethod
    def backward(ctx, grad_out):
        g_node, g_tau = ctx.saved_tensors
        return grad_out.to(g_node.dtype) * g_node, grad_out.to(g_tau.dtype) * g_tau, None
