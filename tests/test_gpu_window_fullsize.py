"""The differentiable window at its full configuration: the 256x128 double
Harris sheet with 32 particles per cell per species (2,097,152 particles),
20 FP32 steps with a checkpoint every 5, loss = energy of the k_x = 2 pi/L_x
B_y mode after the window. The gradient in the amplitude of the initial B_y
perturbation from loss.backward() (the chained step adjoints) against a
central difference with h = 1e-3 of the amplitude (0.01).

The mode energy grows as the square of the amplitude while the mode is
linear, so the central difference carries almost no truncation error at
h = 1e-3; FP32 rounding of the loss (~1e-7 of it) puts ~1e-4 of noise on
the difference quotient; the FP32 adjoint agrees with the FP64 oracle's
gradient to 1e-3 on the small window; particles whose trajectories cross
a cell line between the perturbed runs add kinks of the same order. A bound
of 1e-2 leaves room for these.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_window_fullsize_gradient_in_amplitude_matches_central_difference():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    from paper_2509_11100_gb300.window import ModeEnergyWindow, WindowLoss
    from relsim_inputs import HarrisConfig, make_harris
    hc = HarrisConfig(nx=256, ny=128, ppc=32, theta_T=0.3, delta=1.0, sigma=10.0, pert=0.01, dt=0.5)
    st = make_harris(hc)
    d = st["derived"]
    xc = np.arange(hc.nx) + 0.5
    shape = np.zeros((3, hc.ny, hc.nx))
    shape[1] = d["B0"] * np.cos(2 * np.pi * xc / hc.nx)[None, :]
    shape = shape.reshape(3, -1)
    base = st["B"] - hc.pert * shape
    cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=32, gmres_tol=1e-7, gmres_restart=60)
    win = ModeEnergyWindow(cfg, 20, checkpoint_every=5)
    E0 = torch.tensor(st["E"], dtype=torch.float64, requires_grad=True)
    pert = torch.tensor(hc.pert, dtype=torch.float64, requires_grad=True)
    loss = WindowLoss.apply(win, st, E0, pert, base, shape)
    loss.backward()
    h = 1e-3

    def L(p):
        with torch.no_grad():
            return float(WindowLoss.apply(win, st, torch.tensor(st["E"]), torch.tensor(p), base, shape))

    fd = (L(hc.pert + h) - L(hc.pert - h)) / (2 * h)
    g = float(pert.grad)
    win.close()
    print(f"window 256x128: dL/dpert adjoint {g:.6e}, central difference {fd:.6e}, rel {abs(fd - g) / abs(fd):.2e}")
    assert np.isfinite(g) and g > 0
    assert abs(fd - g) < 1e-2 * abs(fd), (fd, g)
