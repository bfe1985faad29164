"""A differentiable window of RelSIM steps on the GPU.

The loss is the energy of Fourier mode m of B_y along x after the last step
of the window (the linear-tearing diagnostic of Sec. 3.1). Gradients with
respect to the initial E field (per node) and B field (per cell centre), and
through B, the amplitude of an initial B_y perturbation, come from one step's
adjoint chained backwards over the window: per step, the pushes' adjoints
(fields fixed), the field adjoint with their dL/dE^{n+theta}, then the
deposits' adjoints (relsim_push_adjoint, relsim_field_adjoint,
relsim_deposit_adjoint). The forward pass keeps a checkpoint of the state
every `checkpoint_every` steps; the backward pass reloads each checkpoint,
recomputes that segment's steps to recover their start states, and runs the
adjoints backwards through it. Particles are matched across the re-sort of
every push by the ids the library carries (`track_ids`).

Everything runs in the library's kernels; this module only orders the
calls and moves the per-step gradients between particle orders. It covers
the base scheme (gbar = gamma(u^n)).
"""
from __future__ import annotations

import numpy as np

from . import RELSIM_ERR_NOT_CONVERGED, Simulation, relsim_config

__all__ = ["ModeEnergyWindow", "mode_energy_and_gradient", "WindowLoss"]


def mode_energy_and_gradient(B, nx, ny, dV, mode=1, component=1):
    """W_m = (1/2) dV (2/nx) sum_j |F_{m,j}|^2 (F the DFT along x of row j of
    B_c, as relsim_field_modes for 0 < m < nx/2) and dW_m/dB, (3, nx*ny)."""
    Bc = np.asarray(B, dtype=np.float64).reshape(3, ny, nx)[component]
    th = 2.0 * np.pi * mode * np.arange(nx) / nx
    Fr = (Bc * np.cos(th)[None, :]).sum(axis=1)
    Fi = -(Bc * np.sin(th)[None, :]).sum(axis=1)
    W = 0.5 * dV * (2.0 / nx) * float(np.sum(Fr * Fr + Fi * Fi))
    g = np.zeros((3, ny, nx))
    g[component] = (2.0 * dV / nx) * (Fr[:, None] * np.cos(th)[None, :] - Fi[:, None] * np.sin(th)[None, :])
    return W, g.reshape(3, nx * ny)


class ModeEnergyWindow:
    """Forward and backward over `nsteps` steps from a state dict (species
    with x, y, ux, uy, uz, w; E; B) on one context (cfg.track_ids is set)."""

    def __init__(self, cfg: relsim_config, nsteps: int, checkpoint_every: int = 5, mode: int = 1,
                 stream=None):
        if cfg.gamma_pred:
            raise ValueError("the window's adjoint covers the base scheme (gamma_pred = 0)")
        cfg.track_ids = 1
        self.cfg = cfg
        self.nsteps = int(nsteps)
        self.every = max(1, int(checkpoint_every))
        self.mode = mode
        self.sim = Simulation(cfg, stream)
        self.nx, self.ny = cfg.nx, cfg.ny
        self.nsp = cfg.nspecies
        self.dV = cfg.dx * cfg.dy
        self.checkpoints = {}
        self.iters = []

    def close(self):
        self.sim.close()

    # -- state transfer ---------------------------------------------------
    def _state(self):
        """The current state as host arrays in the library's current order."""
        sp = []
        for s in range(self.nsp):
            x, u, w, ids = self.sim.particles(s, ids=True)
            sp.append({"x": x, "u": u, "w": w, "ids": ids})
        E, B = self.sim.fields()
        return {"species": sp, "E": E, "B": B}

    def _load(self, st):
        """Load a state; the ids restart at the load order (which it keeps:
        the particles are already in cell order)."""
        for s, sp in enumerate(st["species"]):
            self.sim.load_species(s, sp["x"], sp["u"], sp["w"])
        self.sim.set_fields(st["E"], st["B"])

    def _step(self):
        led, code = self.sim.step(ledger=True)
        if code not in (0, RELSIM_ERR_NOT_CONVERGED):
            raise RuntimeError(f"step failed: {code}")
        self.iters.append(led["gmres_iters"])

    # -- forward ------------------------------------------------------------
    def forward(self, state):
        """Run the window from `state` (a relsim_inputs-style dict); keep a
        checkpoint every `checkpoint_every` steps; return the loss."""
        init = {"species": [{"x": np.stack([np.asarray(sp["x"], np.float64), np.asarray(sp["y"], np.float64)], 1),
                             "u": np.stack([np.asarray(sp[k], np.float64) for k in ("ux", "uy", "uz")], 1),
                             "w": np.asarray(sp["w"], np.float64)} for sp in state["species"]],
                "E": np.asarray(state["E"], np.float64), "B": np.asarray(state["B"], np.float64)}
        self._load(init)
        self.checkpoints = {}
        for n in range(self.nsteps):
            if n % self.every == 0:
                self.checkpoints[n] = self._state()
            self._step()
        E, B = self.sim.fields()
        self.loss, self.gB_final = mode_energy_and_gradient(B, self.nx, self.ny, self.dV, self.mode)
        return self.loss

    # -- backward -----------------------------------------------------------
    def _step_adjoint(self, pre, gpart, gE1, gB1):
        """Reload the step's start state, rebuild and solve, run the three
        adjoints. gpart[s] = (gu1 (n, 3), gx1 (n, 2)) in the start state's
        order; returns the gradients with respect to the start state (per
        species, in its order), dL/dE^n and dL/dB^n."""
        self._load(pre)
        self.sim.build()
        self.sim.solve()
        gp = [self.sim.push_adjoint(s, gpart[s][0], gpart[s][1]) for s in range(self.nsp)]
        gEt = sum(g["E"] for g in gp)
        gf = self.sim.field_adjoint(gE1, gB1, gEt=gEt)
        gd = [self.sim.deposit_adjoint(s, gf["J"], gf["M"]) for s in range(self.nsp)]
        gB = gf["B0"] + sum(g["B"] for g in gp) + sum(g["B"] for g in gd)
        gsp = [(gp[s]["u"] + gd[s]["u"], gp[s]["x"] + gd[s]["x"]) for s in range(self.nsp)]
        return gsp, gf["E0"], gB

    def backward(self):
        """dL/dE and dL/dB of the window's initial fields (3, ncell) each, and
        per species the gradients (du (N, 3), dx (N, 2)) of the initial
        particles, indexed by their order in the initial state."""
        nx, ny = self.nx, self.ny
        gE = np.zeros((3, nx * ny))
        gB = self.gB_final.copy()
        # per species, gradients indexed by the particles' initial ids
        gid = [(np.zeros((len(sp["w"]), 3)), np.zeros((len(sp["w"]), 2)))
               for sp in self.checkpoints[0]["species"]]
        starts = sorted(self.checkpoints)
        for k in range(len(starts) - 1, -1, -1):
            s0 = starts[k]
            s1 = starts[k + 1] if k + 1 < len(starts) else self.nsteps
            ck = self.checkpoints[s0]
            # recompute the segment's start states; their ids count from the
            # checkpoint's load, mapped back to initial ids through it
            pres = [ck]
            self._load(ck)
            for n in range(s0, s1 - 1):
                self._step()
                st = self._state()
                for s in range(self.nsp):
                    st["species"][s]["ids"] = ck["species"][s]["ids"][st["species"][s]["ids"]]
                pres.append(st)
            for n in range(s1 - 1, s0 - 1, -1):
                pre = pres[n - s0]
                gpart = []
                for s in range(self.nsp):
                    ids = pre["species"][s]["ids"]
                    gpart.append((gid[s][0][ids], gid[s][1][ids]))
                gsp, gE, gB = self._step_adjoint(pre, gpart, gE, gB)
                for s in range(self.nsp):
                    ids = pre["species"][s]["ids"]
                    gid[s][0][ids] = gsp[s][0]
                    gid[s][1][ids] = gsp[s][1]
        self.grad_particles = gid
        return {"E": gE, "B": gB, "particles": gid}


def _torch():
    import torch
    return torch


class WindowLoss:
    """torch.autograd.Function over a ModeEnergyWindow: loss = energy of the
    B_y mode after the window, as a function of the initial E (3, ncell) and
    the amplitude `pert` of a B_y perturbation pert * shape added to a base B
    (shape: (3, ncell)). Built lazily so that importing the package does not
    import torch."""

    _fn = None

    @classmethod
    def apply(cls, window: ModeEnergyWindow, state: dict, E0, pert, B_base, B_shape):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, E0t, pertt, win, st, Bb, Bs):
                    st2 = dict(st)
                    st2["E"] = E0t.detach().cpu().double().numpy()
                    st2["B"] = np.asarray(Bb, np.float64) + float(pertt) * np.asarray(Bs, np.float64)
                    loss = win.forward(st2)
                    ctx.win, ctx.Bs = win, np.asarray(Bs, np.float64)
                    return torch.tensor(loss, dtype=torch.float64)

                @staticmethod
                def backward(ctx, gout):
                    g = ctx.win.backward()
                    gE = torch.from_numpy(g["E"]) * gout
                    gp = torch.tensor(float(np.sum(g["B"] * ctx.Bs)), dtype=torch.float64) * gout
                    return gE, gp, None, None, None, None

            cls._fn = _F
        return cls._fn.apply(E0, pert, window, state, B_base, B_shape)
