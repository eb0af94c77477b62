"""Physics through the CUDA path: the Langmuir oscillation of a quiet-start
plasma (Appendix A set-up, omega_p dt = 0.1, k = 2 pi) oscillates at the
least-damped root of the Vlasov-Poisson dispersion relation, in every
precision and re-binning scheme and on the 3D brick path.  The reference
frequency is the kinetic root (k lambda_D = 0.314), 3.4% above Bohm-Gross."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)


def kinetic_root(klam):
    """Least-damped root of 1 + (1 + zeta Z(zeta)) / (k lambda_D)^2 = 0,
    zeta = omega / (sqrt 2 k v_th), Z from scipy's Faddeeva function."""
    sp = pytest.importorskip("scipy.special")
    opt = pytest.importorskip("scipy.optimize")

    def F(vv):
        w = vv[0] + 1j * vv[1]
        z = w / (math.sqrt(2) * klam)
        r = 1 + (1 + z * 1j * math.sqrt(math.pi) * sp.wofz(z)) / klam ** 2
        return [r.real, r.imag]

    return opt.fsolve(F, [math.sqrt(1 + 3 * klam ** 2), -0.01])[0]


def measure_omega(g, w, steps, t0):
    """Mode-k amplitude of the deposited charge at every step, fitted by a
    damped cosine after t0."""
    from scipy.optimize import curve_fit
    pos = g.vertex_table()
    M = 3 ** int(g.info().depth)
    ph = np.exp(-2j * np.pi * w.k_mode * pos[0] / M)
    amps = []
    for _ in range(steps):
        amps.append(float((g.deposit() * ph).sum().real))
        g.step(w.dt)
    tt = np.arange(steps) * w.dt
    m = tt >= t0
    f = lambda t, a, om, p, gm: a * np.cos(om * t + p) * np.exp(gm * t)
    popt, _ = curve_fit(f, tt[m], np.array(amps)[m], p0=[amps[0], 1.15, 0.0, 0.0])
    return abs(popt[1])


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_langmuir_frequency_2d(scheme, precision):
    pytest.importorskip("scipy")
    w = W.langmuir(2, 3, 64, vth=0.05)
    g = pic.Pic(2, w.flags, w.x, w.v, scheme=scheme, precision=precision, q=w.q, qm=w.qm, ion=w.ion,
                sweeps=400, omega=1.0)
    g.init_leapfrog(w.dt)
    om = measure_omega(g, w, 200, 6.0)
    target = kinetic_root(2 * math.pi * 0.05)
    assert abs(om / target - 1) < 0.02, (om, target)
    assert g.stats().error == 0


def test_langmuir_frequency_3d_brick_path():
    """27^3 leaves, 8 particles per cell, FP32 split, PIT: the brick kernels."""
    pytest.importorskip("scipy")
    w = W.langmuir(3, 3, 8, vth=0.05)
    g = pic.Pic(3, w.flags, w.x, w.v, scheme=pic.PIT, precision=pic.FP32_SPLIT, q=w.q, qm=w.qm, ion=w.ion,
                sweeps=400, omega=1.0, track_ids=False)
    assert g.info().brick == 1
    g.init_leapfrog(w.dt)
    om = measure_omega(g, w, 200, 6.0)
    target = kinetic_root(2 * math.pi * 0.05)
    assert abs(om / target - 1) < 0.03, (om, target)
    assert g.stats().error == 0


@pytest.mark.parametrize("d,depth,ppc", [(2, 3, 16), (3, 3, 8)])
def test_split_precision_error_per_result(d, depth, ppc):
    """FP32 split (int32 leaf + FP32 offset) against FP64 on the GPU after 50
    steps of the Langmuir set-up, per result: deposited density, field,
    positions and velocities (the same errors as the two oracles give:
    about 2e-6 relative for density and field, 3e-7 L for positions)."""
    w = W.langmuir(d, depth, ppc, vth=0.05)
    kw = dict(scheme=pic.PIT, q=w.q, qm=w.qm, ion=w.ion, sweeps=50, omega=0.8)
    a = pic.Pic(d, w.flags, w.x, w.v, precision=pic.FP64, **kw)
    b = pic.Pic(d, w.flags, w.x, w.v, precision=pic.FP32_SPLIT, **kw)
    for g in (a, b):
        g.init_leapfrog(w.dt)
    for _ in range(50):
        a.step(w.dt)
        b.step(w.dt)
    rel = lambda x, y: float(np.max(np.abs(x - y)) / np.max(np.abs(y)))
    assert rel(b.deposit(), a.deposit()) < 1e-5
    assert rel(b.field(), a.field()) < 1e-5
    xa, va = a.particles()
    xb, vb = b.particles()
    ia, ib = np.argsort(a.bins()[1]), np.argsort(b.bins()[1])
    dx = np.abs(xa[:, ia] - xb[:, ib])
    dx = np.minimum(dx, 1.0 - dx)
    assert dx.max() < 2e-6
    assert rel(vb[:, ib], va[:, ia]) < 5e-6


def test_split_precision_frequency():
    """Measured Langmuir frequency, FP32 split against FP64 (same workload):
    within 0.1% of each other."""
    pytest.importorskip("scipy")
    w = W.langmuir(2, 3, 64, vth=0.05)
    om = []
    for prec in (pic.FP64, pic.FP32_SPLIT):
        g = pic.Pic(2, w.flags, w.x, w.v, scheme=pic.PIT, precision=prec, q=w.q, qm=w.qm, ion=w.ion,
                    sweeps=400, omega=1.0)
        g.init_leapfrog(w.dt)
        om.append(measure_omega(g, w, 200, 6.0))
    assert abs(om[1] / om[0] - 1) < 1e-3, om
