"""Test helpers: build the product solver and the oracle from the same Case."""
import numpy as np

import oracle
from paper_2609_24785_b300 import lee, workloads


# one line per measured parity result, printed in pytest's terminal summary
PARITY_LOG = []


def log_result(line):
    PARITY_LOG.append(line)
    print(line)


def make_solver(case, precision="fp64", bind=True, probe_capacity=None, tile=None):
    s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision=precision,
                   periodic_x=case.periodic[0], periodic_y=case.periodic[1])
    workloads.apply_to(case, s)
    if tile:
        s.set_tile(*tile)
    if len(case.probes):
        s.set_probes(case.probes, probe_capacity or max(case.steps, 1))
    s.plan()
    if bind:
        s.bind()
        workloads.apply_state(case, s)
    return s


def make_oracle(case, probe_capacity=None, f32_storage=False):
    o = oracle.Oracle(case.nx, case.ny, case.h, case.cfl, periodic_x=case.periodic[0], periodic_y=case.periodic[1])
    if f32_storage:
        o.set_f32_storage(True)
    workloads.apply_to(case, o)
    o.setup()
    if len(case.probes):
        o.set_probes(case.probes, probe_capacity or max(case.steps, 1))
    workloads.apply_state(case, o)
    return o


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0))


def field_error(s, o, fluid=None):
    """rel-L2 over the fluid nodes of (p, u, v) stacked."""
    if fluid is None:
        fluid = o.kind() == 1
    a = np.concatenate([s.field(f)[fluid] for f in range(3)])
    b = np.concatenate([o.field(f)[fluid] for f in range(3)])
    return rel_l2(a, b)
