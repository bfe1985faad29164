"""A differentiable window of RelSIM steps on the GPU.

The loss is the energy of Fourier mode m of B_y along x after the last step
of the window (the linear-tearing diagnostic of Sec. 3.1). Gradients with
respect to the initial E field (per node) and B field (per cell centre), and
through B, the amplitude of an initial B_y perturbation, come from one
step's adjoint chained backwards over the window (relsim_step_adjoint: the
pushes' adjoints with the fields fixed, the field adjoint with their
dL/dE^{n+theta}, the deposits' adjoints). The forward pass keeps a
checkpoint of the state every `checkpoint_every` steps in device memory;
the backward pass reloads each checkpoint, recomputes that segment's steps
to recover their start states (kept on the device) and runs the step
adjoints backwards through it. Every particle carries its index in the
initial state as its id (relsim_relabel_particles after each reload), and
the per-particle gradients live in that id order on the device, so no step
needs a reordering or a host transfer.

Everything runs in the library's kernels; this module only orders the
calls. It covers both readings of gbar (gamma(u^n), and with gamma_pred the
predicted gamma(u^n + beta E^n(x)), whose step adjoint also carries dL/dgbar
to E^n, u^n and x).
"""
from __future__ import annotations

import numpy as np

from . import RELSIM_ERR_NOT_CONVERGED, Simulation, relsim_config

__all__ = ["ModeEnergyWindow", "WindowLoss", "parameter_gradient"]


class ModeEnergyWindow:
    """Forward and backward over `nsteps` steps from a state dict (species
    with x, y, ux, uy, uz, w; E; B) on one context (cfg.track_ids is set)."""

    def __init__(self, cfg: relsim_config, nsteps: int, checkpoint_every: int = 5, mode: int = 1,
                 stream=None):
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
        self.adjoint_iters = []

    def close(self):
        self.checkpoints = {}
        self.sim.close()

    # -- state transfer (device to device) ----------------------------------
    def _state(self):
        """The current state as CUDA tensors in the library's current order;
        the ids are the particles' indices in the initial state."""
        sp = []
        for s in range(self.nsp):
            x, u, w, ids = self.sim.particles(s, ids=True, device=True)
            sp.append({"x": x, "u": u, "w": w, "ids": ids})
        E, B = self.sim.fields(device=True)
        return {"species": sp, "E": E, "B": B}

    def _load(self, st):
        """Load a saved state and give each particle its saved id."""
        for s, sp in enumerate(st["species"]):
            self.sim.load_species(s, sp["x"], sp["u"], sp["w"])
            self.sim.relabel(s, sp["ids"])
        self.sim.set_fields(st["E"], st["B"])

    def _step(self):
        led, code = self.sim.step(ledger=False)
        if code not in (0, RELSIM_ERR_NOT_CONVERGED):
            raise RuntimeError(f"step failed: {code}")

    # -- forward ------------------------------------------------------------
    def forward(self, state):
        """Run the window from `state` (a relsim_inputs-style dict); keep a
        checkpoint every `checkpoint_every` steps; return the loss."""
        for s, sp in enumerate(state["species"]):
            x = np.stack([np.asarray(sp["x"], np.float64), np.asarray(sp["y"], np.float64)], 1)
            u = np.stack([np.asarray(sp[k], np.float64) for k in ("ux", "uy", "uz")], 1)
            self.sim.load_species(s, x, u, np.asarray(sp["w"], np.float64))   # ids = initial indices
        self.sim.set_fields(np.asarray(state["E"], np.float64), np.asarray(state["B"], np.float64))
        self.checkpoints = {}
        for n in range(self.nsteps):
            if n % self.every == 0:
                self.checkpoints[n] = self._state()
            self._step()
        # the loss and its gradient in B^N, on the device
        e, self.gB_final = self.sim.field_mode_gradient(1, self.mode, device=True)
        self.loss = float(e.item())
        return self.loss

    # -- backward -----------------------------------------------------------
    def backward(self):
        """dL/dE and dL/dB of the window's initial fields (3, ncell) each, and
        per species the gradients (du (N, 3), dx (N, 2)) of the initial
        particles, indexed by their order in the initial state (host arrays)."""
        import torch
        dev = self.checkpoints[0]["E"].device
        gE = torch.zeros((3, self.nx * self.ny), dtype=torch.float64, device=dev)
        gB = self.gB_final.clone()
        gu = [torch.zeros((sp["w"].shape[0], 3), dtype=torch.float64, device=dev)
              for sp in self.checkpoints[0]["species"]]
        gx = [torch.zeros((sp["w"].shape[0], 2), dtype=torch.float64, device=dev)
              for sp in self.checkpoints[0]["species"]]
        gw = [torch.zeros((sp["w"].shape[0],), dtype=torch.float64, device=dev)
              for sp in self.checkpoints[0]["species"]]
        self.adjoint_iters = []
        starts = sorted(self.checkpoints)
        for k in range(len(starts) - 1, -1, -1):
            s0 = starts[k]
            s1 = starts[k + 1] if k + 1 < len(starts) else self.nsteps
            # recompute the segment's start states; the last one stays loaded
            pres = [self.checkpoints[s0]]
            self._load(pres[0])
            for n in range(s0, s1 - 1):
                self._step()
                if n < s1 - 2:
                    pres.append(self._state())
            for n in range(s1 - 1, s0 - 1, -1):
                if n < s1 - 1:
                    self._load(pres[n - s0])
                it, _, _ = self.sim.step_adjoint(gE, gB, gu, gx, gw)
                self.adjoint_iters.append(it)
        torch.cuda.synchronize(dev)
        gid = [(gu[s].cpu().numpy(), gx[s].cpu().numpy()) for s in range(self.nsp)]
        self.grad_particles = gid
        return {"E": gE.cpu().numpy(), "B": gB.cpu().numpy(), "particles": gid,
                "w": [gw[s].cpu().numpy() for s in range(self.nsp)]}


def parameter_gradient(grads, state_minus, state_plus, h, jump=1e-3):
    """dL/dp for a parameter p of the initial state (e.g. the sheet
    thickness of the loader), pathwise: the window's gradients (backward()'s
    output, particles in the state's order) contracted with the central
    difference (state_plus - state_minus)/(2h) of two states built at p - h
    and p + h from the same random numbers, over E, B and every particle's
    position, momentum and weight. A particle whose momentum changes by more
    than `jump` between the two states took a different discrete choice in
    the loader (a sheet membership or a flip) and is left out; jump=None
    keeps every particle (a loader with no discrete choice, e.g. the
    weighted Harris loading). Returns (dL/dp, number of particles left
    out)."""
    g = float(np.sum(grads["E"] * (np.asarray(state_plus["E"]) - np.asarray(state_minus["E"]))))
    g += float(np.sum(grads["B"] * (np.asarray(state_plus["B"]) - np.asarray(state_minus["B"]))))
    out = 0
    for s, (sm, sp) in enumerate(zip(state_minus["species"], state_plus["species"])):
        gu, gx = grads["particles"][s]
        gw = grads["w"][s]
        du = np.stack([np.asarray(sp[k]) - np.asarray(sm[k]) for k in ("ux", "uy", "uz")], axis=1)
        dx = np.stack([np.asarray(sp[k]) - np.asarray(sm[k]) for k in ("x", "y")], axis=1)
        dw = np.asarray(sp["w"]) - np.asarray(sm["w"])
        keep = np.ones(dw.shape, bool) if jump is None else np.abs(du).max(axis=1) <= jump
        out += int((~keep).sum())
        g += float(np.sum(gu[keep] * du[keep]) + np.sum(gx[keep] * dx[keep]) + np.sum(gw[keep] * dw[keep]))
    return g / (2.0 * h), out


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
