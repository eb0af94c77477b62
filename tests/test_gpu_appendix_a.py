"""The validation run of Appendix A through the CUDA path: a thermal plasma at
rest on a 243 x 243 grid (cell = Debye length), 100 particles per cell at
random positions, v_th = 1, q/m = -1, omega_p dt = 0.01, the potential sampled
every 150 steps.  The random start seeds Langmuir waves at every wave vector;
the space-time Fourier transform of the potential must put their power on the
Vlasov-Poisson dispersion relation: along the k_2 = 0 cut (and k_1 = 0) the
frequency of the spectral peak follows the least-damped kinetic root of
1 + (1 + zeta Z(zeta)) / (k lambda_D)^2 = 0 (Bohm-Gross, omega^2 = 1 + 3 k^2
lambda_D^2, in the long-wave limit), and at omega = 1.14 the power sits on the
ring of wave vectors of that frequency.

The particle step (deposit, gather, push, re-bin) runs in the library's
kernels; the field solve goes through the solve hook: the periodic bilinear
finite-element Poisson problem solved exactly in Fourier space (the library's
built-in Jacobi sweeps cannot follow the long waves of a 243^2 grid), the
vertex field by the library's central differences."""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

D2D = 3  # cudaMemcpyDeviceToDevice


def kinetic_root(klam):
    """Least-damped root (real part) of the Langmuir branch."""
    sp = pytest.importorskip("scipy.special")
    opt = pytest.importorskip("scipy.optimize")

    def F(vv):
        w = vv[0] + 1j * vv[1]
        z = w / (math.sqrt(2) * klam)
        r = 1 + (1 + z * 1j * math.sqrt(math.pi) * sp.wofz(z)) / klam ** 2
        return [r.real, r.imag]

    return opt.fsolve(F, [math.sqrt(1 + 3 * klam ** 2), -0.01])[0]


class SpectralSolve:
    """Solve hook: b = Q - mean(Q), V = b / lambda(theta) mode by mode with the
    symbol of the periodic bilinear stiffness stencil (8/3 at the vertex, -1/3
    at its eight neighbours), E = -(V(+1) - V(-1)) / (2h) per axis.  Every
    copy and kernel is enqueued on the library's stream."""

    def __init__(self, g, M, dtype):
        self.lib = g.lib
        self.lib.cudaMemcpyAsync.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]
        self.lib.cudaMemcpyAsync.restype = C.c_int
        pos = g.vertex_table()                       # vertex -> (ix, iy)
        self.M, self.nv, self.dtype = M, g.n_vertices, dtype
        self.flat = torch.tensor(pos[1] * M + pos[0], device="cuda")
        th = 2 * math.pi * torch.fft.fftfreq(M, device="cuda", dtype=torch.float64)
        cx, cy = torch.cos(th)[None, :], torch.cos(th)[:, None]
        lam = 8.0 / 3 - (2.0 / 3) * (cx + cy) - (4.0 / 3) * cx * cy
        lam[0, 0] = 1.0
        self.inv = 1.0 / lam
        self.inv[0, 0] = 0.0
        self.h = 1.0 / M
        self.samples = []
        self.q = torch.empty(self.nv, dtype=dtype, device="cuda")
        self.e = torch.empty((2, self.nv), dtype=dtype, device="cuda")
        self.keep = False
        self.fn = pic.SOLVE_FN(self)

    def __call__(self, user, Q, E, nv, precision, stream):
        es = torch.cuda.ExternalStream(stream)
        nb = self.q.element_size() * self.nv
        if self.lib.cudaMemcpyAsync(self.q.data_ptr(), Q, nb, D2D, stream):
            return 1
        with torch.cuda.stream(es):
            grid = torch.zeros(self.M * self.M, dtype=torch.float64, device="cuda")
            grid[self.flat] = self.q.double()
            b = grid.view(self.M, self.M)
            b = b - b.mean()
            V = torch.fft.ifft2(torch.fft.fft2(b) * self.inv).real
            Ex = -(torch.roll(V, -1, 1) - torch.roll(V, 1, 1)) / (2 * self.h)
            Ey = -(torch.roll(V, -1, 0) - torch.roll(V, 1, 0)) / (2 * self.h)
            self.e[0] = Ex.reshape(-1)[self.flat].to(self.dtype)
            self.e[1] = Ey.reshape(-1)[self.flat].to(self.dtype)
            if self.keep:
                self.samples.append(V.float().clone())
        if self.lib.cudaMemcpyAsync(E, self.e.data_ptr(), 2 * nb, D2D, stream):
            return 1
        return 0


def spectrum(samples, dt_s):
    """|V(k_1, k_2, omega)|^2 with a Hann window in time (sample mean removed)."""
    Vt = np.stack(samples)
    F = np.fft.fft2(Vt, axes=(1, 2))
    F = F - F.mean(axis=0, keepdims=True)
    win = np.hanning(len(samples))[:, None, None]
    P = np.abs(np.fft.fft(F * win, axis=0)) ** 2
    om = 2 * np.pi * np.fft.fftfreq(len(samples), dt_s)
    return P, om


def peak(om, p, lo, hi):
    """Frequency of the largest power in [lo, hi], refined by a parabola
    through the three bins around it."""
    sel = np.flatnonzero((om >= lo) & (om <= hi))
    i = sel[np.argmax(p[sel])]
    if 0 < i < len(p) - 1 and om[i - 1] < om[i] < om[i + 1]:
        a, b, c = p[i - 1], p[i], p[i + 1]
        den = a - 2 * b + c
        off = 0.5 * (a - c) / den if den != 0 else 0.0
        return om[i] + off * (om[i + 1] - om[i])
    return om[i]


def test_langmuir_dispersion_appendix_a():
    pytest.importorskip("scipy")
    w = W.thermal_plasma(2, 5, 100, dt=0.01, seed=5)
    M = 3 ** 5
    stream = torch.cuda.Stream()
    g = pic.Pic(2, w.flags, w.x, w.v, scheme=pic.PIT, precision=pic.FP32_SPLIT, q=w.q, qm=w.qm, ion=w.ion,
                sweeps=0, track_ids=False, stream=stream)
    del w.x, w.v
    solve = SpectralSolve(g, M, torch.float32)
    g.init_leapfrog(w.dt, solve.fn)
    every, n_samples = 150, 160                     # sampling period 1.5 / omega_p, T = 240 / omega_p
    for i in range(every * n_samples):
        solve.keep = i % every == 0
        g.step(w.dt, solve.fn)
    g.sync()
    torch.cuda.synchronize()
    assert not g.stats().error
    P, om = spectrum([s.cpu().numpy() for s in solve.samples], every * w.dt)
    T = len(om)
    half = T // 2
    omp = om[1:half]                                # positive frequencies; bin i pairs with T - i
    dom = om[1] - om[0]
    rows = []
    for m in range(2, 12):                          # k lambda_D = 2 pi m / 243 = 0.05 ... 0.28
        klam = 2 * math.pi * m / M
        # k along x and along y, both signs of k and of omega
        p = P[:, 0, m] + P[:, 0, -m] + P[:, m, 0] + P[:, -m, 0]
        pp = p[1:half] + p[T - 1:T - half:-1]
        w_peak = peak(omp, pp, 0.8, 2.0)
        rows.append((m, klam, w_peak, kinetic_root(klam), math.sqrt(1 + 3 * klam ** 2)))
    print("m  k lambda_D  omega_peak  kinetic  Bohm-Gross")
    for r in rows:
        print("%2d  %.4f  %.4f  %.4f  %.4f" % r)
    for m, klam, wp, wk, wbg in rows:
        assert abs(wp - wk) <= max(0.03, 1.2 * dom), (m, klam, wp, wk)
    # the (k_1, k_2) cut at omega = 1.14: the power of each |k| shell; its
    # maximum sits at the wave number whose kinetic root is 1.14
    i114 = 1 + int(np.argmin(np.abs(omp - 1.14)))
    ring = P[i114] + P[T - i114]
    kk = np.fft.fftfreq(M) * M
    kr = np.sqrt(kk[None, :] ** 2 + kk[:, None] ** 2)
    shells = np.array([ring[(kr >= s - 0.5) & (kr < s + 0.5)].mean() for s in range(1, 15)])
    s_max = 1 + int(np.argmax(shells))
    k_expect = min(range(1, 15), key=lambda s: abs(kinetic_root(2 * math.pi * s / M) - om[i114]))
    print("omega cut %.3f: shell of largest power %d, expected %d" % (om[i114], s_max, k_expect))
    assert abs(s_max - k_expect) <= 1
