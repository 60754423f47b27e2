"""Dual adaptive explicit time integration (Section 2), written step by step.

Notation follows Section 2:

* Strang splitting of Eq. 2 over one step dt: step I (diffusion, dt/2), step II
  (reaction, dt), step III (diffusion, dt/2).  Steps III and I of consecutive
  steps together form "step B"; step II is "step A".  Here one call of
  ``Simulation.step`` runs I, II, III in order, which is the same sequence of
  sub-steps as the merged form.
* Step A: forward Euler (Rush-Larsen gates for TP06) with dt_ar = dt / k,
  k = k0 + floor(|dV/dt|), k0 = 5 if dV/dt > 0 else 1, clamped to
  [1, k_max], k_max = floor(dt / dt0).
* Steps I/III: forward Euler with dt_ad = dt / (2 l) on M_L dV/dt = -K V,
  l = floor(dt / (2 dt_s)) if dt/2 > dt_s else 1, dt_s from Eq. 3.

Readings where Section 2 is silent (each is listed with its reason in the
design notes of the repository):

* R-k:   dV/dt "at the previous iteration" is (V(t_n) - V(t_{n-1})) / dt, the
         rate of the split solution over the previous step, V(t_n) being the
         solution at the synchronisation time between the two diffusion
         halves; at t_0 the rate is 0 (k = 1).  k is fixed per node for the
         whole step A.
* R-dt0: k_max = floor(dt / dt0 + 1e-9) with dt0 = 0.01 ms.
* R-stim: a stimulus is on at sub-step start time t when
         t0 + p T - 1e-9 <= t < t0 + p T + dur - 1e-9 for some p < count.
* R-LAT: activation time = first upward crossing of v_th between two
         synchronisation times, linearly interpolated; -1 if never.
* R-OSTAR: OSTAR uses dt' = dt / ceil(dt / dt_s) when dt_s < dt, l = 1;
         OST uses the given dt with k = l = 1.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cells as _cells
from . import fem as _fem

EPS_T = 1e-9


def gershgorin_dt(K, m, safety=0.9):
    """Eq. 3: dt_s = 0.9 min_i m_ii / (k_ii + sum_{j != i} |k_ij|)."""
    K = sp.csr_matrix(K)
    diag = K.diagonal()
    absrow = np.asarray(abs(K).sum(axis=1)).ravel()
    off = absrow - np.abs(diag)
    denom = diag + off
    with np.errstate(divide="ignore"):
        ratio = np.where(denom > 0, m / np.where(denom > 0, denom, 1.0), np.inf)
    return safety * float(ratio.min())


def lambda_max(K, m):
    """Largest eigenvalue of M_L^-1 K (= that of the symmetric M^-1/2 K M^-1/2)."""
    s = 1.0 / np.sqrt(m)
    C = sp.diags(s) @ sp.csr_matrix(K) @ sp.diags(s)
    n = C.shape[0]
    if n <= 400:
        return float(np.linalg.eigvalsh(C.toarray()).max())
    val = spla.eigsh(C, k=1, which="LA", return_eigenvectors=False, tol=1e-12, maxiter=20000)
    return float(val[0])


def l_rule(dt, dt_s, rounding="floor"):
    """Section 2: l = floor(dt / (2 dt_s)) if dt/2 > dt_s, else 1 (ceil as an option)."""
    if dt / 2.0 > dt_s:
        x = dt / (2.0 * dt_s)
        return int(math.floor(x)) if rounding == "floor" else int(math.ceil(x))
    return 1


def k_max_rule(dt, dt0):
    return max(1, int(math.floor(dt / dt0 + 1e-9)))


def k_rule(rate_mv_per_ms, k_max):
    """k = k0 + floor(|dV/dt|), k0 = 5 for dV/dt > 0 else 1, capped at k_max."""
    r = np.asarray(rate_mv_per_ms, dtype=np.float64)
    k0 = np.where(r > 0.0, 5, 1)
    a = np.minimum(np.abs(r), 1e6)
    k = k0 + np.floor(a).astype(np.int64)
    return np.minimum(k, k_max).astype(np.int64)


def stimulus_on(stim, t):
    """Boolean (per entry of t) for one stimulus (R-stim)."""
    t = np.asarray(t, dtype=np.float64)
    on = np.zeros(t.shape, dtype=bool)
    for p in range(int(stim.count)):
        t0 = stim.t_start + p * stim.period
        on |= (t >= t0 - EPS_T) & (t < t0 + stim.duration - EPS_T)
    return on


class Simulation:
    """The split scheme on one tissue, plain and unfused (FP64)."""

    def __init__(self, K, m, model, stimuli=(), dt=0.1, dt0=0.01, scheme="daeti",
                 l_round="floor", v_threshold=None, gate_rl=True, state0=None, k_rule="total"):
        self.K = sp.csr_matrix(K)
        self.m = np.asarray(m, dtype=np.float64)
        self.n_nodes = self.K.shape[0]
        self.model = model
        self.stimuli = list(stimuli)
        self.scheme = scheme
        self.gate_rl = gate_rl
        self.dt_s = gershgorin_dt(self.K, self.m)
        dt = float(dt)
        if scheme == "daeti":
            self.l = l_rule(dt, self.dt_s, l_round)
            self.k_max = k_max_rule(dt, dt0)
            self.adaptive_k = True
        elif scheme == "ostar":
            if self.dt_s < dt:
                dt = dt / math.ceil(dt / self.dt_s - 1e-12)
            self.l = 1
            self.k_max = k_max_rule(dt, dt0)
            self.adaptive_k = True
        elif scheme == "ost":
            self.l = 1
            self.k_max = 1
            self.adaptive_k = False
        else:
            raise ValueError(scheme)
        self.dt = dt
        self.dt_ad = dt / (2.0 * self.l)
        self.v_th = v_threshold
        self.S = model.initial_state(self.n_nodes) if state0 is None else np.array(state0, dtype=np.float64)
        self.n = 0
        self.v_sync = self.S[0].copy()          # V(t_{n-1}) at the last synchronisation
        self.k = np.ones(self.n_nodes, dtype=np.int64)
        # dV/dt of the k rule (reading R-k): "total", the split solution's
        # (V(t_n) - V(t_{n-1}))/dt; "reaction" (reading R-k2), the reaction's
        # dV/dt at each node's last sub-step of the previous step II (0 at t_0)
        if k_rule not in ("total", "reaction"):
            raise ValueError(k_rule)
        self.k_rule = k_rule
        self.rrate = np.zeros(self.n_nodes)
        self.act = np.full(self.n_nodes, -1.0)
        self.minv = 1.0 / self.m
        self._members = []
        for st in self.stimuli:
            mask = np.zeros(self.n_nodes, dtype=bool)
            mask[np.asarray(st.nodes, dtype=np.int64)] = True
            self._members.append(mask)

    # -- step I / III -----------------------------------------------------------
    def diffuse(self, n_sub):
        V = self.S[0]
        for _ in range(n_sub):
            V = V - self.dt_ad * self.minv * (self.K @ V)
        self.S[0] = V

    # -- step II ---------------------------------------------------------------
    def stimulus_current(self, idx, t_sub):
        J = np.zeros(len(idx))
        for st, mask in zip(self.stimuli, self._members):
            J += np.where(mask[idx] & stimulus_on(st, t_sub), st.amplitude, 0.0)
        return J

    def react(self):
        t_n = self.n * self.dt
        k = self.k
        for s in range(int(k.max())):
            idx = np.nonzero(k > s)[0]
            dt_ar = self.dt / k[idx]
            t_sub = t_n + s * dt_ar
            J = self.stimulus_current(idx, t_sub)
            sub = self.S[:, idx]
            model = self.model.for_nodes(idx) if isinstance(self.model, _cells.TP06) else self.model
            if self.k_rule == "reaction":
                last = k[idx] == s + 1          # nodes taking their last sub-step
                self.rrate[idx[last]] = model.dvdt(sub, J)[last]
            if isinstance(self.model, _cells.TP06):
                self.S[:, idx] = model.substep(sub, dt_ar, J, gate_rl=self.gate_rl)
            else:
                self.S[:, idx] = model.substep(sub, dt_ar, J)

    # -- synchronisation at t_{n+1} ----------------------------------------------
    def sync(self):
        V = self.S[0]
        if self.v_th is not None:
            t_prev = (self.n - 1) * self.dt
            up = (self.act < 0.0) & (self.v_sync < self.v_th) & (V >= self.v_th)
            frac = (self.v_th - self.v_sync[up]) / (V[up] - self.v_sync[up])
            self.act[up] = t_prev + self.dt * frac
        if self.k_rule == "reaction":
            rate = self.rrate * self.model.vscale
        else:
            rate = (V - self.v_sync) / self.dt * self.model.vscale
        self.k = k_rule(rate, self.k_max) if self.adaptive_k else np.ones(self.n_nodes, dtype=np.int64)
        self.v_sync = V.copy()

    def step(self):
        self.diffuse(self.l)        # step I  (dt/2)
        self.react()                # step II (dt)
        self.diffuse(self.l)        # step III (dt/2)
        self.n += 1
        self.sync()

    def run(self, n_steps, snapshot_every=0, callback=None):
        snaps = []
        for _ in range(int(n_steps)):
            self.step()
            if snapshot_every and self.n % snapshot_every == 0:
                snaps.append(self.S[0].copy())
            if callback is not None:
                callback(self)
        return snaps

    @property
    def t(self):
        return self.n * self.dt


def simulation_from_workload(wl, scheme="daeti", dt=None, l_round="floor", gate_rl=True, k_rule="total"):
    """Assemble K, m and build a ``Simulation`` for an ``inputs.Workload``."""
    K, m = _fem.assemble_workload(wl)
    model = _cells.make_model(wl.model, wl.model_params, getattr(wl, "cell_type", None))
    return Simulation(K, m, model, wl.stimuli, dt=wl.dt if dt is None else dt, dt0=wl.dt0,
                      scheme=scheme, l_round=l_round, v_threshold=wl.v_threshold, gate_rl=gate_rl,
                      k_rule=k_rule)
