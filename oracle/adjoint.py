"""Discrete adjoint of the split step for the Mitchell-Schaeffer model (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The forward map is the scheme of ``oracle.scheme.Simulation`` (Section 2):
per step, l diffusion sub-steps v <- (I - dt_ad M^-1 K) v, the reaction with k
forward-Euler sub-steps, l diffusion sub-steps, then the synchronisation.  The
discrete choices of the scheme -- k per node and step (Section 2's rule) and
the Mitchell-Schaeffer gate branch v < v_gate per sub-step -- are recorded in
the unperturbed forward run and held fixed ("frozen schedule"); the gradient
is that of the resulting smooth map.  ``forward(replay=...)`` reruns with a
recorded schedule so that central differences see the same map.

Loss: L = sum over samples j and sensors s of (v_s(t_j) - d_js)^2, samples at
the synchronisation times t = j * sample_every * dt.

Parameters: isotropic element conductivities D_e (K = sum_e D_e K_e with K_e
the element stiffness for unit D), and tau_close.  With nodal values, D_e is
the mean of the element's nodes (reading R-D).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import cells as _cells
from . import fem as _fem
from . import scheme as _scheme


class MSAdjointGrid:
    """Structured 2D/3D grid, isotropic per-element D, Mitchell-Schaeffer cells."""

    def __init__(self, dim, n, h, d_elem, ms_params, stimuli, dt=0.1, dt0=0.01, l_override=None):
        self.dim, self.n, self.h = dim, tuple(n), float(h)
        self.conn = _fem.grid_elements(dim, n)
        self.n_nodes = int(np.prod(n[:dim]))
        Kref, Mref = _fem.box_element_matrices(dim, h, np.eye(dim))
        self.Kref = Kref
        self.m = np.zeros(self.n_nodes)
        np.add.at(self.m, self.conn, Mref.sum(axis=1)[None, :])
        self.ms_params = tuple(float(p) for p in ms_params)
        self.stimuli = list(stimuli)
        self.dt, self.dt0 = float(dt), float(dt0)
        self.set_d(d_elem, l_override)

    def assemble(self, d_elem):
        nl = self.conn.shape[1]
        vals = (np.asarray(d_elem)[:, None, None] * self.Kref[None]).ravel()
        rows = np.repeat(self.conn, nl, axis=1).ravel()
        cols = np.tile(self.conn, (1, nl)).ravel()
        K = sp.csr_matrix((vals, (rows, cols)), shape=(self.n_nodes, self.n_nodes))
        K.sum_duplicates()
        return K

    def set_d(self, d_elem, l_override=None):
        self.d_elem = np.asarray(d_elem, dtype=np.float64).copy()
        self.K = self.assemble(self.d_elem)
        self.dt_s = _scheme.gershgorin_dt(self.K, self.m)
        self.l = l_override if l_override is not None else _scheme.l_rule(self.dt, self.dt_s)
        self.dt_ad = self.dt / (2.0 * self.l)
        self.k_max = _scheme.k_max_rule(self.dt, self.dt0)

    # ---------------------------------------------------------------- forward
    def forward(self, n_steps, sensors, sample_every, data=None, tau_close=None, replay=None, keep=False):
        """Run n_steps; returns (loss, record).  ``record`` holds the schedule and,
        with keep=True, every intermediate needed by the reverse sweep."""
        p = list(self.ms_params)
        if tau_close is not None:
            p[3] = float(tau_close)
        model = _cells.MitchellSchaeffer(*p)
        sim = _scheme.Simulation(self.K, self.m, model, self.stimuli, dt=self.dt, dt0=self.dt0)
        sim.l, sim.dt_ad = self.l, self.dt_ad
        n = self.n_nodes
        rec = {"k": [], "branch": [], "steps": []}
        loss = 0.0
        samples = []
        for step in range(n_steps):
            st = {}
            # step I
            v = sim.S[0].copy()
            d1 = []
            for _ in range(self.l):
                d1.append(v.copy())
                v = v - self.dt_ad * (self.K @ v) / self.m
            sim.S[0] = v
            # step II with frozen k and branches
            k = replay["k"][step] if replay is not None else sim.k.copy()
            rec["k"].append(k.copy())
            v, hh = sim.S[0].copy(), sim.S[1].copy()
            st["react_in"] = (v.copy(), hh.copy())
            t_n = sim.n * self.dt
            br_step = np.zeros((int(k.max()), n), dtype=bool)
            for s in range(int(k.max())):
                idx = np.nonzero(k > s)[0]
                dt_ar = self.dt / k[idx]
                J = sim.stimulus_current(idx, t_n + s * dt_ar)
                vi, hi = v[idx], hh[idx]
                if replay is not None:
                    low = replay["branch"][step][s, idx]
                else:
                    low = vi < model.v_gate
                br_step[s, idx] = low
                dv = hi * vi * vi * (1.0 - vi) / model.tau_in - vi / model.tau_out + J
                dh = np.where(low, (1.0 - hi) / model.tau_open, -hi / model.tau_close)
                v[idx] = vi + dt_ar * dv
                hh[idx] = hi + dt_ar * dh
            rec["branch"].append(br_step)
            sim.S[0], sim.S[1] = v, hh
            # step III
            v = sim.S[0].copy()
            d2 = []
            for _ in range(self.l):
                d2.append(v.copy())
                v = v - self.dt_ad * (self.K @ v) / self.m
            sim.S[0] = v
            sim.n += 1
            sim.sync()
            if replay is not None and step + 1 < n_steps:
                sim.k = replay["k"][step + 1]
            if (step + 1) % sample_every == 0:
                vs = v[sensors].copy()
                samples.append(vs)
                if data is not None:
                    loss += float(np.sum((vs - data[len(samples) - 1]) ** 2))
            if keep:
                st["d1"], st["d2"], st["v_end"] = d1, d2, v.copy()
                rec["steps"].append(st)
        rec["samples"] = np.array(samples)
        rec["model"] = model
        return loss, rec

    # ---------------------------------------------------------------- reverse
    def gradient(self, n_steps, sensors, sample_every, data, tau_close=None):
        """Loss, dL/dD_e (per element) and dL/dtau_close by the discrete adjoint."""
        loss, rec = self.forward(n_steps, sensors, sample_every, data, tau_close, keep=True)
        model = rec["model"]
        n = self.n_nodes
        lam_v = np.zeros(n)
        lam_h = np.zeros(n)
        g_d = np.zeros(len(self.d_elem))
        g_tau = 0.0
        n_samples = n_steps // sample_every
        conn = self.conn

        def d_grad(mu_out, v_in):
            # v_out = v_in - dt_ad M^-1 K v_in:  dL/dD_e += -dt_ad mu_out^T K_e v_in
            return -self.dt_ad * np.einsum("ea,ab,eb->e", mu_out[conn], self.Kref, v_in[conn])

        for step in range(n_steps - 1, -1, -1):
            st = rec["steps"][step]
            if (step + 1) % sample_every == 0:
                j = (step + 1) // sample_every - 1
                if j < n_samples:
                    lam_v[sensors] += 2.0 * (st["v_end"][sensors] - data[j])
            # step III transposed: lambda_in = (I - dt_ad K M^-1) lambda_out
            for v_in in reversed(st["d2"]):
                mu = lam_v / self.m
                g_d += d_grad(mu, v_in)
                lam_v = lam_v - self.dt_ad * (self.K @ mu)
            # step II transposed, sub-step by sub-step from the recorded inputs
            k = rec["k"][step]
            br = rec["branch"][step]
            v, hh = st["react_in"][0].copy(), st["react_in"][1].copy()
            t_n = step * self.dt
            traj = []
            for s in range(int(k.max())):
                idx = np.nonzero(k > s)[0]
                dt_ar = self.dt / k[idx]
                J = self._stim(idx, t_n + s * dt_ar)
                vi, hi = v[idx], hh[idx]
                traj.append((idx, dt_ar, vi.copy(), hi.copy(), br[s, idx]))
                low = br[s, idx]
                dv = hi * vi * vi * (1.0 - vi) / model.tau_in - vi / model.tau_out + J
                dh = np.where(low, (1.0 - hi) / model.tau_open, -hi / model.tau_close)
                v[idx] = vi + dt_ar * dv
                hh[idx] = hi + dt_ar * dh
            for idx, dt_ar, vi, hi, low in reversed(traj):
                fv = hi * (2.0 * vi - 3.0 * vi * vi) / model.tau_in - 1.0 / model.tau_out
                fh = vi * vi * (1.0 - vi) / model.tau_in
                gh = np.where(low, -1.0 / model.tau_open, -1.0 / model.tau_close)
                lv, lh = lam_v[idx], lam_h[idx]
                g_tau += float(np.sum(np.where(low, 0.0, lh * dt_ar * hi / model.tau_close ** 2)))
                lam_v[idx] = (1.0 + dt_ar * fv) * lv
                lam_h[idx] = dt_ar * fh * lv + (1.0 + dt_ar * gh) * lh
            # step I transposed
            for v_in in reversed(st["d1"]):
                mu = lam_v / self.m
                g_d += d_grad(mu, v_in)
                lam_v = lam_v - self.dt_ad * (self.K @ mu)
        return loss, g_d, g_tau, rec

    def _stim(self, idx, t_sub):
        J = np.zeros(len(idx))
        for st in self.stimuli:
            mask = np.zeros(self.n_nodes, dtype=bool)
            mask[np.asarray(st.nodes, dtype=np.int64)] = True
            J += np.where(mask[idx] & _scheme.stimulus_on(st, t_sub), st.amplitude, 0.0)
        return J


def element_d_from_nodes(conn, d_node):
    """D_e = mean of the element's nodal values (reading R-D)."""
    return np.asarray(d_node)[conn].mean(axis=1)


def nodal_gradient(conn, g_elem, n_nodes):
    """Chain rule of ``element_d_from_nodes``."""
    g = np.zeros(n_nodes)
    np.add.at(g, conn, (np.asarray(g_elem) / conn.shape[1])[:, None])
    return g
