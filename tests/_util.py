"""Shared helpers for the GPU parity tests: run the same seeded inputs through the
CUDA library and through the oracle, and compare what must be identical."""
import numpy as np

from paper_1909_00709_gb300 import inputs


def event_key_gpu(e):
    return (int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]))


def event_key_orc(e):
    return (int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]))


def gpu_context(abi, shapes, seeds, **opt):
    temps, powers, coeffs = [], [], []
    for s, seed in zip(shapes, seeds):
        t, p = inputs.grid_inputs(*s, seed=seed)
        temps.append(t)
        powers.append(p)
        coeffs.append(inputs.hotspot_coeffs(*s))
    return abi.Context(shapes, temps, powers, coeffs, **opt)


def oracle_run(orc, shape, seed, steps, mode, flips=None, **kw):
    co = inputs.hotspot_coeffs(*shape)
    temp, power = inputs.grid_inputs(*shape, seed=seed)
    st = orc.Stencil(shape, orc.hotspot_points(co))
    C = orc.source_term(power, co)
    return orc.run(st, C, temp, steps, mode, flips, **kw)


def rel_err(gpu, ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(np.asarray(gpu, dtype=np.float64) - ref) / np.abs(ref)))


def compare_events(gpu_ev, orc_res, grid=0):
    """Event sets must be identical outside the (step, plane) pairs the oracle marks
    as marginal (residual within 5 % of the threshold)."""
    marg = orc_res["marginal"]
    g = {event_key_gpu(e) for e in gpu_ev if int(e["grid"]) == grid}
    o = {event_key_orc(e) for e in orc_res["events"]}
    g = {k for k in g if (k[0], k[1]) not in marg}
    o = {k for k in o if (k[0], k[1]) not in marg}
    return g, o
