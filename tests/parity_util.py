"""Helpers shared by the GPU parity tests: run the CUDA path (through the C ABI
binding) and the CPU oracle on the same seeded workload and collect V
snapshots and activation times."""
import numpy as np

from oracle import scheme


def gpu_available():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def ensure_lib():
    from paper_2011_04747_gb300 import binding, build

    import os

    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


def run_gpu(wl, n_steps, every, **opts):
    binding = ensure_lib()
    s = binding.solver_from_workload(wl, **opts)
    stab = s.daeti_get_stability()
    dt = stab["dt"]
    snaps = []
    n = 0
    while n < n_steps:
        n = min(n + every, n_steps)
        s.daeti_advance(n * dt)
        snaps.append(s.daeti_read_v())
    act = s.daeti_read_activation()
    s.daeti_synchronize()
    state = s.daeti_read_state()
    s.close()
    return np.array(snaps), act, stab, state


def run_oracle(wl, n_steps, every, scheme_name="daeti", dt=None, l_round="floor", gate_rl=True, k_rule="total"):
    sim = scheme.simulation_from_workload(wl, scheme=scheme_name, dt=dt, l_round=l_round, gate_rl=gate_rl,
                                          k_rule=k_rule)
    snaps = []
    n = 0
    while n < n_steps:
        k = min(every, n_steps - n)
        sim.run(k)
        n += k
        snaps.append(sim.S[0].copy())
    return np.array(snaps), sim.act.copy(), sim


def act_error(a, b):
    """max |a - b| over nodes activated in both; also whether the activated sets agree."""
    both = (a >= 0) & (b >= 0)
    same_set = bool(np.array_equal(a >= 0, b >= 0))
    err = float(np.max(np.abs(a[both] - b[both]))) if both.any() else 0.0
    return err, same_set, int(both.sum())
