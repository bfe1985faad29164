"""The differentiable window at its full configuration: the 256x128 double
Harris sheet with 32 particles per cell per species (2,097,152 particles),
20 FP32 steps with a checkpoint every 5, loss = energy of the k_x = 2 pi/L_x
B_y mode after the window (Sec. 3.1's tearing diagnostic). Three gradients
from one backward pass (the chained step adjoints) against central
differences of the whole window with h = 1e-3:

* the amplitude of the initial B_y perturbation (0.01), through
  loss.backward() of the torch.autograd.Function, with either reading of
  gbar;
* the sheet half-thickness delta of the loader, pathwise (the window's
  gradients in the initial fields, momenta, positions and weights contracted
  with the loader's central difference at delta -+ h, same random numbers),
  on the weighted loading of the sheet, whose particles are smooth in delta
  (the sampled loading draws sheet membership and flips the boost: at
  h = 1e-3 those discrete choices change for ~1e3 particles, and their
  jumps add a term of the same order as the pathwise one to the central
  difference, which no pathwise gradient contains);
* the initial E_y at one node.

The FP32 adjoint itself agrees with the FP64 oracle's gradient to ~1e-6 on
the small windows (test_gpu_window.py). What separates it from a central
difference at h = 1e-3 is the difference quotient: FP32 rounding of the
loss (~1e-7 of it) over 2h, the O(h^2) truncation, and the loss being only
piecewise smooth (the shape functions are piecewise linear: a particle whose
trajectory crosses a cell line between the two perturbed runs puts a kink
inside the stencil). The measured agreement is printed; the bounds below
leave room for these effects at this h.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

H = 1e-3


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    from paper_2509_11100_gb300.window import ModeEnergyWindow
    from relsim_inputs import HarrisConfig, make_harris
    hc = HarrisConfig(nx=256, ny=128, ppc=32, theta_T=0.3, delta=1.0, sigma=10.0, pert=0.01, dt=0.5)
    cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=32, gmres_tol=1e-7, gmres_restart=60)
    win = ModeEnergyWindow(cfg, 20, checkpoint_every=5)
    yield rs, hc, make_harris, HarrisConfig, win
    win.close()


@pytest.mark.parametrize("pred", [0, 1])
def test_window_fullsize_gradient_in_amplitude_matches_central_difference(setup, pred):
    import torch
    from paper_2509_11100_gb300.window import ModeEnergyWindow, WindowLoss
    rs, hc, make_harris, HarrisConfig, win = setup
    if pred:   # the predicted gbar, whose adjoint also runs through E^n and u^n in gbar
        cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=32, gmres_tol=1e-7, gmres_restart=60, gamma_pred=1)
        win = ModeEnergyWindow(cfg, 20, checkpoint_every=5)
    st = make_harris(hc)
    d = st["derived"]
    xc = np.arange(hc.nx) + 0.5
    shape = np.zeros((3, hc.ny, hc.nx))
    shape[1] = d["B0"] * np.cos(2 * np.pi * xc / hc.nx)[None, :]
    shape = shape.reshape(3, -1)
    base = st["B"] - hc.pert * shape
    E0 = torch.tensor(st["E"], dtype=torch.float64, requires_grad=True)
    pert = torch.tensor(hc.pert, dtype=torch.float64, requires_grad=True)
    loss = WindowLoss.apply(win, st, E0, pert, base, shape)
    loss.backward()

    def L(p):
        with torch.no_grad():
            return float(WindowLoss.apply(win, st, torch.tensor(st["E"]), torch.tensor(p), base, shape))

    fd = (L(hc.pert + H) - L(hc.pert - H)) / (2 * H)
    g = float(pert.grad)
    if pred:
        win.close()
    print(f"window 256x128 (gamma_pred={pred}): dL/dpert adjoint {g:.6e}, central difference {fd:.6e}, "
          f"rel {abs(fd - g) / abs(fd):.2e}")
    assert np.isfinite(g) and g > 0
    assert abs(fd - g) < 1e-2 * abs(fd), (fd, g)


def test_window_fullsize_gradient_in_delta_and_one_node_of_E(setup):
    from paper_2509_11100_gb300.window import parameter_gradient
    rs, hc, make_harris, HarrisConfig, win = setup
    cfg = dict(hc.asdict())

    def state(delta):
        c = dict(cfg)
        c["delta"] = delta
        c["loader"] = "weighted"
        return make_harris(HarrisConfig(**c))

    st0, stm, stp = state(hc.delta), state(hc.delta - H), state(hc.delta + H)
    win.forward(st0)
    g = win.backward()
    gd, out = parameter_gradient(g, stm, stp, H, jump=None)
    assert out == 0
    fd = (win.forward(stp) - win.forward(stm)) / (2 * H)
    print(f"window 256x128 (weighted loading): dL/ddelta pathwise {gd:.6e}, "
          f"central difference {fd:.6e}, rel {abs(fd - gd) / abs(fd):.2e}")
    assert np.isfinite(gd) and abs(fd - gd) < 1e-2 * abs(fd), (gd, fd)
    # one node's E_y: the node of largest |dL/dE_y| on the sheet's midplane row
    row = hc.ny // 4
    gy = g["E"][1].reshape(hc.ny, hc.nx)
    i = int(np.argmax(np.abs(gy[row])))
    node = row * hc.nx + i
    stE = dict(st0)
    Ep, Em = np.array(st0["E"]), np.array(st0["E"])
    Ep[1, node] += H
    Em[1, node] -= H
    stE["E"] = Ep
    Lp = win.forward(stE)
    stE["E"] = Em
    Lm = win.forward(stE)
    fdE = (Lp - Lm) / (2 * H)
    ge = float(g["E"][1, node])
    print(f"window 256x128: dL/dE_y at node ({i}, {row}) adjoint {ge:.6e}, central difference {fdE:.6e}, "
          f"rel {abs(fdE - ge) / max(abs(fdE), 1e-300):.2e}")
    assert np.isfinite(ge) and abs(fdE - ge) < 5e-2 * abs(fdE), (ge, fdE)
