"""Builders that set up the same seeded case on the CUDA path and on the oracle.

Each side receives only the arrays from paper_2402_13171_gb300.inputs and
turns them into populations with its own code."""
import numpy as np

import oracle as O
from paper_2402_13171_gb300 import lbm


def gpu_lattice(dom: dict, storage="fp32", diag_every=0, tile=(0, 0)):
    return lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], collision=dom.get("collision", "cumulant"),
                              nu=dom.get("nu", 0.01), smag_c=dom.get("smag_c", 0.0), storage=storage,
                              bc=dom.get("bc", ("periodic",) * 3), body_force=dom.get("body_force", (0, 0, 0)),
                              seed=dom.get("seed", 0), diag_every=diag_every, tile=tile)


def oracle_sim(dom: dict, turbines=()):
    d = O.make_domain(dom["nx"], dom["ny"], dom["nz"], collision=dom.get("collision", "cumulant"),
                      nu=dom.get("nu", 0.01), smag_c=dom.get("smag_c", 0.0), bc=dom.get("bc", ("periodic",) * 3),
                      body_force=dom.get("body_force", (0, 0, 0)), inflow_kind=dom.get("inflow_kind", 0),
                      u_ref=dom.get("u_ref", (0, 0, 0)), z0=dom.get("z0", 0.1), z_ref=dom.get("z_ref", 1.0),
                      noise_rel=dom.get("noise_rel", 0.0), seed=dom.get("seed", 0))
    return O.Sim(d, [O.TurbineSpec(**t) for t in turbines])


def setup_pair(dom: dict, turbines=(), rho=None, u=None, fneq=None, storage="fp32", diag_every=0, tile=(0, 0),
               inflow=False):
    """GPU lattice and oracle run with the same domain, rotors and initial state."""
    g = gpu_lattice(dom, storage=storage, diag_every=diag_every, tile=tile)
    s = oracle_sim(dom, turbines)
    if inflow:
        g.set_inflow(u_ref=dom.get("u_ref", (0, 0, 0)), kind=dom.get("inflow_kind", 0), z0=dom.get("z0", 0.1),
                     z_ref=dom.get("z_ref", 1.0), noise_rel=dom.get("noise_rel", 0.0))
    for t in turbines:
        g.add_turbine(**t)
    if rho is not None or u is not None or fneq is not None or not inflow:
        g.init_fields(rho, u, fneq)
    s.init_fields(rho, u, fneq)
    return g, s


def max_du(g, s):
    _, ug = g.moments()
    _, uo = s.moments()
    return float(np.abs(ug - uo).max())
