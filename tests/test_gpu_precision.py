"""Precision of the FP32 form against the FP64 oracle over a run, per field,
per energy-ledger term and per spectrum bin (the paper's quantities: the
fields of Sec. 2, Table 1's energy error column, the spectra of Sec. 3.2).

Workload: the 64x32 double Harris sheet (16 particles per cell and species,
dt = 0.5, theta = 0.5, GMRES 1e-7 in FP32 and 1e-12 in the oracle), 100
steps from one FP32-representable initial state, once with each reading of
the Lorentz factor in alpha, Jhat, M and the push. Each step records, for
the FP32 GPU run and for an oracle run started from momenta perturbed at the
FP32 rounding level (6e-8, the dynamics' own conditioning), the relative
error against the oracle of
  * E and B (relative L2 norm over the grid),
  * the ledger terms W_E, W_B, K (after the step), the particles' work
    dt sum w q (ubar/gbar).E (against the larger of its value and its RMS
    over the run: a signed flow that passes close to zero on some steps)
    and the relativistic mismatch term,
  * the 256-bin spectrum of gamma - 1 over [1e-2, 1e4] (both species): the
    largest relative error over the bins holding at least 1e-3 of the
    weight, the L1 distance of the weights over all bins, and the particles'
    own divergence eta, the largest relative difference of gamma - 1 between
    the GPU's particle and the oracle's particle of the same id.
A quantity's horizon is the last step up to which its error stays below
1e-5. Orbits in the sheet are chaotic: round-off grows about e-fold per 12
steps, so every horizon is finite; the assertions are the measured horizons
(with a margin) and, at every step, the FP32 field errors within 10x of the
perturbed oracle's, the GPU's spectrum equal to the histogram of its own
particles (bins decided in FP32), and the spectrum's L1 distance within what
the measured divergence allows: a particle changes bin only if an edge lies
within eta (plus FP32 rounding of gamma - 1) of its oracle value, so the L1
distance is at most twice the weight of the oracle's particles that close
to an edge. With RELSIM_REPORT_DIR set, the curves are written there as
JSON.
"""
import json
import os

import numpy as np
import pytest

from relsim_inputs import HarrisConfig, make_harris

pytestmark = pytest.mark.gpu

NX, NY, PPC, DT, NSTEPS = 64, 32, 16, 0.5, 100
EDGES = np.geomspace(1e-2, 1e4, 257)
TERMS = ("W_E", "W_B", "K", "work", "mismatch")


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    return rs


def fp32_state(st):
    for sp in st["species"]:
        for k in ("x", "y"):
            s = np.asarray(sp[k])
            fl = np.floor(s)
            f = (s - fl).astype(np.float32).astype(np.float64)
            f = np.minimum(f, np.float64(np.nextafter(np.float32(1.0), np.float32(0.0))))
            sp[k] = fl + f
        for k in ("ux", "uy", "uz", "w"):
            sp[k] = np.asarray(sp[k]).astype(np.float32).astype(np.float64)
    st["E"] = np.asarray(st["E"]).astype(np.float32).astype(np.float64)
    st["B"] = np.asarray(st["B"]).astype(np.float32).astype(np.float64)
    return st


def oracle_terms(lo):
    return {"W_E": lo["W_E1"], "W_B": lo["W_B1"], "K": lo["K1"], "work": lo["work_particles"],
            "mismatch": lo["mismatch"]}


def gpu_terms(led):
    return {"W_E": led["W_E"], "W_B": led["W_B"], "K": led["K"], "work": led["work_particles"],
            "mismatch": led["mismatch"]}


def oracle_spectrum(orc, P):
    w = np.zeros(258)
    for s in range(2):
        sp = P.species(s)
        w += orc.spectrum(sp["ux"], sp["uy"], sp["uz"], sp["w"], EDGES, 0, precision=64)[0]
    return w


def gamma_minus_one(ux, uy, uz):
    u2 = ux * ux + uy * uy + uz * uz
    return u2 / (np.sqrt(1.0 + u2) + 1.0)


def near_edge_weight(xo, w, eta):
    """Weight of the particles whose gamma - 1 lies within a relative
    distance eta of a bin edge."""
    k = np.clip(np.searchsorted(EDGES, xo), 1, EDGES.size - 1)
    d = np.minimum(np.abs(xo - EDGES[k - 1]), np.abs(EDGES[k] - xo))
    return float(w[d <= eta * xo].sum())


def spectrum_errors(wg, wo):
    sel = wo >= 1e-3 * wo.sum()
    rel = np.abs(wg[sel] - wo[sel]) / wo[sel]
    return float(rel.max()), float(np.abs(wg - wo).sum() / wo.sum())


def horizon(errs, tol=1e-5):
    h = 0
    for n, e in enumerate(errs, start=1):
        if e >= tol:
            break
        h = n
    return h


def run_curves(rs, orc, pred):
    st = fp32_state(make_harris(HarrisConfig(nx=NX, ny=NY, ppc=PPC, dt=DT)))
    sim = rs.Simulation(rs.make_config(NX, NY, dt=DT, precision=32, gmres_tol=1e-7, gamma_pred=pred,
                                       track_ids=True))
    sim.load_state(st)
    c = orc.make_config(NX, NY, dt=DT, gmres_tol=1e-12, gamma_pred=pred)
    P = orc.Particles(st["species"])
    Pp = P.copy()
    rng = np.random.default_rng(1)
    for k in ("ux", "uy", "uz"):
        a = getattr(Pp, k)
        a *= 1.0 + 6e-8 * rng.choice([-1.0, 1.0], size=a.size)
    E, B = st["E"], st["B"]
    Ep, Bp = st["E"], st["B"]
    cur = {k: [] for k in ("E", "B") + TERMS + ("spec_bin_max", "spec_l1", "eta")}
    pert = {k: [] for k in cur}
    l1_bound = []
    raw_work = []   # (oracle, GPU, perturbed oracle) per step
    for n in range(NSTEPS):
        led, status = sim.step(ledger=True)
        assert status == 0
        E, B, lo, _ = orc.step(c, P, E, B)
        Ep, Bp, lp, _ = orc.step(c, Pp, Ep, Bp)
        Eg, Bg = sim.fields()
        nE, nB = np.linalg.norm(E), np.linalg.norm(B)
        cur["E"].append(float(np.linalg.norm(Eg - E) / nE))
        cur["B"].append(float(np.linalg.norm(Bg - B) / nB))
        pert["E"].append(float(np.linalg.norm(Ep - E) / nE))
        pert["B"].append(float(np.linalg.norm(Bp - B) / nB))
        to, tg, tp = oracle_terms(lo), gpu_terms(led), oracle_terms(lp)
        for k in TERMS:
            if k == "work":
                raw_work.append((to[k], tg[k], tp[k]))
                continue
            cur[k].append(abs(tg[k] - to[k]) / abs(to[k]))
            pert[k].append(abs(tp[k] - to[k]) / abs(to[k]))
        wo = oracle_spectrum(orc, P)
        wg = np.zeros(258)
        wp = oracle_spectrum(orc, Pp)
        eta, etap, parts = 0.0, 0.0, []
        for s in range(2):
            wgs, cgs = sim.spectrum(s, EDGES, 0)
            wg += wgs
            _, u, w, ids = sim.particles(s, ids=True)
            order = np.argsort(ids)
            u, w = u[order], w[order]
            # the GPU's spectrum is the histogram of its own particles
            wh, ch = orc.spectrum(u[:, 0], u[:, 1], u[:, 2], w, EDGES, 0, precision=32)
            assert np.array_equal(cgs, ch), (n, s)
            assert np.abs(wgs - wh).max() <= 1e-6 * w.sum()
            o, op = P.species(s), Pp.species(s)
            xo = gamma_minus_one(o["ux"], o["uy"], o["uz"])
            xg = gamma_minus_one(u[:, 0], u[:, 1], u[:, 2])
            xp = gamma_minus_one(op["ux"], op["uy"], op["uz"])
            sel = xo >= 0.5 * EDGES[0]
            eta = max(eta, float((np.abs(xg - xo)[sel] / xo[sel]).max()))
            etap = max(etap, float((np.abs(xp - xo)[sel] / xo[sel]).max()))
            parts.append((xo, o["w"]))
        # a particle may change bin if an edge lies within its divergence:
        # eta (the largest over both species) plus the FP32 rounding of
        # gamma - 1 (a few ulp)
        near = sum(near_edge_weight(xo, w, eta + 1e-6) for xo, w in parts)
        l1_bound.append(2.0 * near / sum(float(w.sum()) for _, w in parts) + 1e-9)
        cur["eta"].append(eta)
        pert["eta"].append(etap)
        cur["spec_bin_max"].append(spectrum_errors(wg, wo)[0])
        cur["spec_l1"].append(spectrum_errors(wg, wo)[1])
        pert["spec_bin_max"].append(spectrum_errors(wp, wo)[0])
        pert["spec_l1"].append(spectrum_errors(wp, wo)[1])
    sim.close()
    # the particles' work is a signed flow that passes close to zero on some
    # steps (there the relative error of the GPU and of the perturbed oracle
    # both jump tenfold); its errors are taken against the larger of its
    # value and its RMS over the run
    w = np.array(raw_work)
    scale = np.maximum(np.abs(w[:, 0]), np.sqrt(np.mean(w[:, 0] ** 2)))
    cur["work"] = [float(v) for v in np.abs(w[:, 1] - w[:, 0]) / scale]
    pert["work"] = [float(v) for v in np.abs(w[:, 2] - w[:, 0]) / scale]
    return cur, pert, l1_bound


# measured horizons (the last step up to which the error stays below 1e-5;
# on GB300: E 37-38, B 63-66, W_E 78-89, W_B 100, K 100, work 54-60 (its
# error against its RMS over the run; against its own value the horizon
# was 4 or 15 from run to run, set by a near-zero work at step 5), mismatch
# 68-69 (gamma(u^n)) and 9 (predicted gamma, a difference of Lorentz
# factors), minus a margin. The spectrum has no 1e-5 horizon: a particle crossing a
# bin edge on one side only moves 2/N of the weight (3e-5 here), so its L1
# distance is held to the perturbed oracle's instead.
MIN_HORIZON = {0: {"E": 30, "B": 50, "W_E": 60, "W_B": 80, "K": 80, "work": 40, "mismatch": 40},
               1: {"E": 30, "B": 50, "W_E": 60, "W_B": 80, "K": 80, "work": 40, "mismatch": 5}}


@pytest.mark.parametrize("pred", [0, 1])
def test_fp32_precision_report(rs, pred):
    import oracle as orc
    cur, pert, l1_bound = run_curves(rs, orc, pred)
    hz = {k: horizon(v) for k, v in cur.items()}
    hzp = {k: horizon(v) for k, v in pert.items()}
    report = {"workload": f"{NX}x{NY} double Harris sheet, {PPC} ppc per species, dt {DT}, {NSTEPS} steps",
              "gamma_bar": "predicted" if pred else "gamma(u^n)",
              "horizon_1e-5": hz, "horizon_1e-5_perturbed_oracle": hzp,
              "fp32_vs_oracle": cur, "perturbed_oracle_vs_oracle": pert,
              "spec_l1_bound_from_eta": l1_bound}
    out = os.environ.get("RELSIM_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, f"precision_fp32_64x32_pred{pred}.json"), "w") as f:
            json.dump(report, f)
    print(f"gamma_pred={pred}: horizons (steps within 1e-5) FP32 {hz}; perturbed oracle {hzp}")
    for k, h in MIN_HORIZON[pred].items():
        assert hz[k] >= h, (k, hz)
    # the fields: at every step within 10x of what a rounding-level
    # perturbation of the oracle's own momenta produces (the growth is the
    # dynamics' own)
    for k in ("E", "B"):
        for n, (e, p) in enumerate(zip(cur[k], pert[k]), start=1):
            assert e <= 10 * max(p, 1e-7), (k, n, e, p)
    # the spectrum: particles cross bin edges one by one as the trajectories
    # separate (the deposit's float atomics make each GPU run's rounding,
    # hence its crossings, differ from run to run); a crossing needs an edge
    # within the particle's divergence
    for n, (e, b) in enumerate(zip(cur["spec_l1"], l1_bound), start=1):
        assert e <= b, ("spec_l1", n, e, b)
