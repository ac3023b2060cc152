"""Pins of the FP64 oracle against things other than itself: a dense solve of the discrete
system, the continuum curl-curl operator (symbolic), closed forms (plane wave, dyadic
Green's function), reciprocity, finite differences and the convergence invariant."""
from __future__ import annotations

import numpy as np
import pytest
import sympy as sp

from oracle import cbs_oracle as co
from oracle import dense, dyadic

LAM = 1.0


def _lossy_grid(nx=8, ny=6, nz=10, ppl=6):
    return co.Grid(nx, ny, nz, LAM / ppl, LAM, 1.0)


def test_discrete_curl_curl_is_real_and_symmetric():
    """C = F^-1 D F is real and symmetric on even and odd lengths (needed by the adjoint)."""
    C = dense.curl_curl_matrix(4, 3, 6, LAM / 4)
    assert np.max(np.abs(C.imag)) < 1e-9 * np.max(np.abs(C))
    assert np.max(np.abs(C - C.T)) < 1e-9 * np.max(np.abs(C))


def test_dense_lippmann_schwinger_matches_cbs_fixed_point():
    """The series converges to the solution of (curl curl - k^2) E = S built as an explicit
    matrix from 1D DFT matrices (no FFT, no Green's function) and solved by LU."""
    g = _lossy_grid()
    rng = np.random.default_rng(1)
    k2 = g.k_vac ** 2 * (1.0 + rng.uniform(0, 1.25, g.shape) + 0.3j)
    S = co.point_source(g, (3, 2, 5), (1.0, 0.5j, 0.2)) + 0.1 * co.plane_wave_source(g, (0.0, 1.0, 0.0), 7)
    res = co.cbs_solve(g, k2, S, tol=1e-13)
    Ed = dense.solve(g.nx, g.ny, g.nz, g.pitch, k2, S)
    assert np.linalg.norm(res.E - Ed) / np.linalg.norm(Ed) < 1e-11


def test_dense_solve_with_absorbing_layers():
    """Same pin with the absorbing layers supplying the loss (real permittivity inside)."""
    g = co.Grid(8, 8, 9, LAM / 4, LAM, 1.0, (2, 2, 2), (2, 1, 2))
    rng = np.random.default_rng(2)
    eps = 1.0 + rng.uniform(0, 1.0, g.shape)
    k2 = co.k_squared(g, eps)
    S = co.point_source(g, (4, 4, 4), (0.0, 1.0, 0.0))
    res = co.cbs_solve(g, k2, S, tol=1e-9, max_iter=200000)
    Ed = dense.solve(g.nx, g.ny, g.nz, g.pitch, k2, S)
    assert np.linalg.norm(res.E - Ed) / np.linalg.norm(Ed) < 1e-6


def test_green_operator_inverts_symbolic_curl_curl():
    """G (curl curl - kt2) E = E for a periodic trigonometric field whose curl curl is taken
    symbolically (sympy), covering transverse and longitudinal parts."""
    g = co.Grid(12, 10, 14, LAM / 5, LAM, 1.0)
    Lx, Ly, Lz = g.nx * g.pitch, g.ny * g.pitch, g.nz * g.pitch
    x, y, z = sp.symbols("x y z", real=True)
    ax, ay, az = 2 * sp.pi / Lx, 2 * sp.pi / Ly, 2 * sp.pi / Lz
    F = sp.Matrix([sp.sin(ax * x) * sp.cos(2 * ay * y) + sp.cos(az * z),
                   sp.cos(ax * x + 3 * az * z) * sp.sin(ay * y),
                   sp.sin(2 * ax * x) + sp.cos(ay * y) * sp.sin(az * z)])

    def curl(V):
        return sp.Matrix([sp.diff(V[2], y) - sp.diff(V[1], z),
                          sp.diff(V[0], z) - sp.diff(V[2], x),
                          sp.diff(V[1], x) - sp.diff(V[0], y)])

    CC = sp.simplify(curl(curl(F)))
    X = np.arange(g.nx) * g.pitch
    Y = np.arange(g.ny) * g.pitch
    Z = np.arange(g.nz) * g.pitch
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    ev = lambda e: np.broadcast_to(sp.lambdify((x, y, z), e, "numpy")(Xg, Yg, Zg), g.shape)
    E = np.stack([ev(F[i]) for i in range(3)]).astype(np.complex128)
    CCE = np.stack([ev(CC[i]) for i in range(3)]).astype(np.complex128)
    kt2 = complex(1.3 * g.k_vac ** 2, 0.7 * g.k_vac ** 2)
    back = co.green_apply(g, kt2, CCE - kt2 * E)
    assert np.linalg.norm(back - E) / np.linalg.norm(E) < 1e-12


def test_homogeneous_absorbing_medium_exact_solution():
    """Constant complex k^2 with a non-trivial splitting (k0^2, epsilon chosen by hand): the
    series converges to the exact periodic solution E = IFFT[G_k2(p) FFT S], independent of
    the splitting."""
    g = _lossy_grid(10, 12, 8)
    k2c = g.k_vac ** 2 * complex(1.4, 0.5)
    k2 = np.full(g.shape, k2c)
    rng = np.random.default_rng(3)
    S = rng.standard_normal((3,) + g.shape) + 1j * rng.standard_normal((3,) + g.shape)
    split = co.Splitting(k0sq=1.1 * g.k_vac ** 2, epsilon=0.9 * g.k_vac ** 2)
    assert split.epsilon >= abs(k2c - split.k0sq)
    res = co.cbs_solve(g, k2, S, tol=1e-13, split=split)
    exact = co.green_apply(g, k2c, S)
    assert np.linalg.norm(res.E - exact) / np.linalg.norm(exact) < 1e-11


def test_series_contracts_on_the_convergence_circle():
    """Eigenvalues of G(p): transverse 1/(|p|^2 - kt2) (twice) and longitudinal -1/kt2 lie on
    the circle |z - i/(2 eps)| = 1/(2 eps) that the convergence proof needs; checked on the
    3x3 blocks recovered from green_apply by unit impulses in k-space."""
    g = co.Grid(6, 5, 4, LAM / 4, LAM, 1.0)
    kt2 = complex(2.0 * g.k_vac ** 2, 1.5 * g.k_vac ** 2)
    eps = kt2.imag
    n = g.n_vox
    rng = np.random.default_rng(4)
    for _ in range(6):
        kz, ky, kx = rng.integers(0, g.nz), rng.integers(0, g.ny), rng.integers(0, g.nx)
        Gm = np.zeros((3, 3), dtype=complex)
        for b in range(3):
            Xh = np.zeros((3,) + g.shape, dtype=complex)
            Xh[b, kz, ky, kx] = 1.0
            Y = co.green_apply(g, kt2, np.fft.ifftn(Xh, axes=(1, 2, 3)))
            Gm[:, b] = np.fft.fftn(Y, axes=(1, 2, 3))[:, kz, ky, kx]
        lam = np.linalg.eigvals(Gm)
        assert np.allclose(np.abs(lam - 0.5j / eps), 0.5 / eps, rtol=1e-10)
        assert n > 0


def test_plane_wave_amplitude_and_phase():
    """Laterally periodic grid, absorbing layers along z: the current sheet launches
    pol exp(i k |z - z_s|) with unit amplitude (checked from 8 voxels past the sheet, where
    the band-limited sheet has rung down)."""
    zpad = 24
    g = co.Grid(8, 8, 96, LAM / 6, LAM, 1.0, (0, 0, zpad), (0, 0, zpad))
    res = co.forward(g, np.ones(g.shape), co.plane_wave_source(g, (1.0, 0.0, 0.0)), tol=1e-9, max_iter=50000)
    z = np.arange(zpad + 8, g.nz - zpad)
    Ex = res.E[0, z, 3, 5]
    ratio = Ex / np.exp(1j * g.k_vac * (z - zpad) * g.pitch)
    assert np.max(np.abs(ratio - 1.0)) < 1.5e-3
    assert np.max(np.abs(res.E[1:])) == 0.0


@pytest.mark.slow
def test_point_dipole_matches_closed_form_dyadic_green():
    """Unit dipole in vacuum inside absorbing layers three wavelengths thick: the field at
    1.25 - 2.75 wavelengths matches G(R) p, off the coordinate planes through the source
    (where the one-voxel source rings), to 1 %."""
    n, ppl, pad = 48, 4, 12
    g = co.Grid(n, n, n, LAM / ppl, LAM, 1.0, (pad,) * 3, (pad,) * 3)
    c = n // 2
    p = np.array([1.0, 0.3, 0.2])
    res = co.forward(g, np.ones(g.shape), co.point_source(g, (c, c, c), p / g.pitch ** 3), tol=1e-6, max_iter=20000)
    zz, yy, xx = np.meshgrid(*[np.arange(pad, n - pad)] * 3, indexing="ij")
    q = np.stack([xx, yy, zz], -1).reshape(-1, 3)
    Rv = (q - c) * g.pitch
    R = np.linalg.norm(Rv, axis=1)
    m = (R >= 1.25) & (R < 2.75) & np.all(np.abs(q - c) >= 2, axis=1)
    Ec = dyadic.dipole_field(g.k_vac, (0, 0, 0), p, Rv[m])
    qm = q[m]
    Eo = np.stack([res.E[k, qm[:, 2], qm[:, 1], qm[:, 0]] for k in range(3)], 1)
    assert np.linalg.norm(Eo - Ec) / np.linalg.norm(Ec) < 1e-2
    # wrong time convention (incoming waves) is far off
    Ein = np.conj(dyadic.dipole_field(g.k_vac, (0, 0, 0), p, Rv[m]))
    assert np.linalg.norm(Eo - Ein) / np.linalg.norm(Ein) > 0.5


def test_dyadic_closed_form_solves_the_wave_equation():
    """curl curl (G p) - k^2 G p = 0 away from the source, by central differences."""
    k = 2 * np.pi
    p = np.array([0.3, -1.0, 0.7])
    h = 1e-3
    for r in ([0.7, 0.2, -0.4], [1.3, -0.9, 0.5]):
        r = np.array(r)

        def E(pt):
            return dyadic.dipole_field(k, (0, 0, 0), p, np.array([pt]))[0]

        # curl curl = grad div - laplacian
        lap = sum((E(r + h * e) - 2 * E(r) + E(r - h * e)) / h ** 2 for e in np.eye(3))
        grad_div = np.zeros(3, dtype=complex)
        for i, ei in enumerate(np.eye(3)):
            for j, ej in enumerate(np.eye(3)):
                d2 = (E(r + h * ei + h * ej)[j] - E(r + h * ei - h * ej)[j]
                      - E(r - h * ei + h * ej)[j] + E(r - h * ei - h * ej)[j]) / (4 * h * h)
                grad_div[i] += d2
        resid = grad_div - lap - k * k * E(r)
        assert np.linalg.norm(resid) < 1e-4 * k * k * np.linalg.norm(E(r))


def _lossy_k2(g, eps, loss=0.3):
    return g.k_vac ** 2 * (eps + 1j * loss)


def test_reciprocity_of_point_sources():
    """A is complex symmetric: E_j of a source along i at r1, seen at r2, equals E_i of a source
    along j at r2, seen at r1 (inhomogeneous lossy medium; even and odd axis lengths)."""
    g = co.Grid(20, 18, 21, LAM / 6, LAM, 1.0)
    rng = np.random.default_rng(5)
    eps = 1.0 + rng.uniform(0, 1.2, g.shape)
    k2 = _lossy_k2(g, eps, 0.4)
    r1, r2 = (6, 7, 8), (13, 9, 14)
    for i, j in ((0, 1), (2, 0), (1, 1)):
        e_i = np.eye(3)[i]
        e_j = np.eye(3)[j]
        a = co.cbs_solve(g, k2, co.point_source(g, r1, e_i), tol=1e-11).E[j, r2[2], r2[1], r2[0]]
        b = co.cbs_solve(g, k2, co.point_source(g, r2, e_j), tol=1e-11).E[i, r1[2], r1[1], r1[0]]
        assert abs(a - b) <= 1e-8 * abs(a)


def test_adjoint_gradient_matches_central_differences():
    """dL/d eps_r at random voxels from one forward and one adjoint solve equals central
    finite differences of L = |E(r0)|^2 (step 1e-4 in eps_r, residual 1e-12), in a lossy
    inhomogeneous medium k^2 = k_vac^2 (eps_r + 0.3 i)."""
    g = co.Grid(16, 14, 18, LAM / 6, LAM, 1.0)
    rng = np.random.default_rng(6)
    eps = 1.0 + rng.uniform(0, 1.25, g.shape)
    S = co.plane_wave_source(g, z_plane=2)
    r0 = (8, 7, 13)
    kw = dict(tol=1e-12, max_iter=200000)
    fwd = co.cbs_solve(g, _lossy_k2(g, eps), S, **kw)
    adj = co.cbs_solve(g, _lossy_k2(g, eps), co.adjoint_source(g, fwd.E, r0), **kw)
    grad = co.gradient(g, fwd.E, adj.E)
    h = 1e-4
    for _ in range(8):
        v = (rng.integers(0, g.nx), rng.integers(0, g.ny), rng.integers(0, g.nz))
        ep, em = eps.copy(), eps.copy()
        ep[v[2], v[1], v[0]] += h
        em[v[2], v[1], v[0]] -= h
        Lp = co.objective(co.cbs_solve(g, _lossy_k2(g, ep), S, **kw).E, r0)
        Lm = co.objective(co.cbs_solve(g, _lossy_k2(g, em), S, **kw).E, r0)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[v[2], v[1], v[0]]) <= 1e-5 * abs(fd) + 1e-8 * np.abs(grad).max()


def test_splitting_and_layer_profile():
    """k0^2 halves the range of Re k^2; epsilon bounds |k^2 - k0^2| with equality somewhere;
    the layer ramp is zero inside, quadratic, and reaches sigma_max on the outer face, where
    the weak-absorption round trip through the layer attenuates by 1e4."""
    g = co.Grid(10, 12, 14, LAM / 8, LAM, 1.0, (2, 3, 4), (3, 2, 4))
    rng = np.random.default_rng(7)
    eps = 1.0 + rng.uniform(0, 1.25, g.shape)
    k2 = co.k_squared(g, eps)
    sp_ = co.splitting(k2)
    assert np.isclose(sp_.k0sq, 0.5 * (k2.real.min() + k2.real.max()))
    dev = np.abs(k2 - sp_.k0sq)
    assert np.isclose(dev.max(), sp_.epsilon) and np.all(dev <= sp_.epsilon * (1 + 1e-15))
    s = co.axis_profile(g, g.nz, 4, 4)
    smax = co.layer_strength(g, 4)
    assert np.all(s[4:-4] == 0) and np.isclose(s[0], smax) and np.isclose(s[-1], smax)
    assert np.isclose(s[2], smax * (2 / 4) ** 2)
    # round trip: 2 * integral of k_vac sigma / (2 n_bg) over the layer = ln(1e4)
    L = 4 * g.pitch
    t = np.linspace(0, 1, 20001)
    integral = np.trapezoid(g.k_vac * smax * t ** 2 / 2.0, t) * L
    assert np.isclose(2 * integral, np.log(1e4), rtol=1e-6)


def test_absorption_maps_each_axis_profile_and_adds_them_in_edges_and_corners():
    """sigma(r) of a grid whose six faces all have different layer widths: a voxel inside one
    layer only gets that axis' ramp at its depth, an edge voxel the sum of two, a corner
    voxel the sum of three (an x/y/z mix-up, a low/high mix-up or a max rule fails here).
    Expected values are layer_strength(L) (t/L)^2 written out per voxel: depth t counts 1 at
    the innermost layer voxel and L on the outer face."""
    g = co.Grid(20, 24, 28, LAM / 8, LAM, 1.0, (2, 3, 4), (5, 6, 7))
    sig = co.absorption(g)      # (nz, ny, nx)
    S = co.layer_strength

    def at(x, y, z):
        return sig[z, y, x]

    # interior: nothing
    assert at(10, 12, 14) == 0.0
    # x only: low face width 2 (x = 0 is depth 2), high face width 5 (x = 19 is depth 5)
    assert np.isclose(at(0, 12, 14), S(g, 2) * (2 / 2) ** 2)
    assert np.isclose(at(1, 12, 14), S(g, 2) * (1 / 2) ** 2)
    assert np.isclose(at(17, 12, 14), S(g, 5) * (3 / 5) ** 2)
    # y only: low width 3, high width 6 (y = 23 is depth 6, y = 18 depth 1)
    assert np.isclose(at(10, 1, 14), S(g, 3) * (2 / 3) ** 2)
    assert np.isclose(at(10, 18, 14), S(g, 6) * (1 / 6) ** 2)
    assert at(10, 17, 14) == 0.0 and at(10, 3, 14) == 0.0
    # z only: low width 4, high width 7 (z = 21 is depth 1)
    assert np.isclose(at(10, 12, 2), S(g, 4) * (2 / 4) ** 2)
    assert np.isclose(at(10, 12, 21), S(g, 7) * (1 / 7) ** 2)
    assert at(10, 12, 20) == 0.0 and at(10, 12, 4) == 0.0
    # edge (x low, z high): the two ramps add
    assert np.isclose(at(0, 12, 27), S(g, 2) + S(g, 7))
    # corner (x high depth 2, y low depth 3, z low depth 1): all three add
    want = S(g, 5) * (2 / 5) ** 2 + S(g, 3) * (3 / 3) ** 2 + S(g, 4) * (1 / 4) ** 2
    assert np.isclose(at(16, 0, 3), want)
    # the strengths differ per width, so the checks above separate the axes
    assert len({round(S(g, L), 9) for L in (2, 3, 4, 5, 6, 7)}) == 6


def _layer_reflection(ppl, layer_wl, round_trip, power, n_bg=1.0):
    """|reflected / incident| amplitude of a plane wave hitting the high-z layer of a 1-voxel
    column (nx = ny = 1: the problem is one-dimensional), fitted as A e^{ik_b z} + B e^{-ik_b z}
    between the source sheet and the layer."""
    L = int(round(layer_wl * ppl))
    nz = 2 * L + 6 * ppl
    g = co.Grid(1, 1, nz, LAM / ppl, LAM, n_bg, (0, 0, L), (0, 0, L), round_trip=round_trip, power=power)
    eps = np.full(g.shape, n_bg ** 2)
    zs = L + 2
    r = co.forward(g, eps, co.plane_wave_source(g, z_plane=zs), tol=1e-11, max_iter=400000)
    E = r.E[0, :, 0, 0]
    z = np.arange(zs + ppl, nz - L - ppl)
    kb = g.k_vac * n_bg
    M = np.stack([np.exp(1j * kb * (z - zs) * g.pitch), np.exp(-1j * kb * (z - zs) * g.pitch)], 1)
    A, B = np.linalg.lstsq(M, E[z], rcond=None)[0]
    return abs(B / A), co.splitting(co.k_squared(g, eps)).epsilon / g.k_vac ** 2


@pytest.mark.parametrize("round_trip,power,n_bg", [(1e-4, 2.0, 1.0), (1e-3, 3.0, 1.0), (1e-2, 2.0, 1.0),
                                                   (1e-3, 2.0, 1.5)])
def test_thick_layer_reflects_its_round_trip(round_trip, power, n_bg):
    """A layer six wavelengths thick (the paper's z layers) reflects a normally incident plane
    wave by about the round-trip amplitude its strength is set for: the reflection there is the
    wave that crossed the layer, met the periodic wrap and came back, and the ramp is gentle
    enough to reflect less.  This pins sigma_max = (p + 1) n_bg ln(1/round_trip) / (k_vac L) --
    the exponent factor and the background index included -- to a measured quantity."""
    refl, _ = _layer_reflection(8, 6, round_trip, power, n_bg)
    assert 0.5 * round_trip <= refl <= 1.6 * round_trip, refl


def test_thin_layer_reflection_and_the_gentler_setting():
    """A layer one wavelength thick (the paper's x and y layers) reflects through its gradient
    more than its round trip: about 5 % for the default 1e-4, while a 1e-2 layer reflects
    less (under 3 %) and halves the series' shift epsilon."""
    r_def, e_def = _layer_reflection(8, 1, 1e-4, 2.0)
    r_gen, e_gen = _layer_reflection(8, 1, 1e-2, 2.0)
    assert 0.02 <= r_def <= 0.07, r_def
    assert r_gen <= 0.03 and r_gen < r_def, (r_gen, r_def)
    assert abs(e_gen / e_def - 0.5) < 0.05, (e_gen, e_def)


def test_corner_rule_max_takes_the_largest_profile():
    g = co.Grid(20, 24, 28, LAM / 8, LAM, 1.0, (2, 3, 4), (5, 6, 7), corner="max")
    sig = co.absorption(g)
    S = co.layer_strength
    want = max(S(g, 5) * (2 / 5) ** 2, S(g, 3) * (3 / 3) ** 2, S(g, 4) * (1 / 4) ** 2)
    assert np.isclose(sig[3, 0, 16], want)
    assert np.isclose(sig[27, 12, 0], max(S(g, 2), S(g, 7)))
    assert np.isclose(sig[14, 12, 0], S(g, 2)) and sig[14, 12, 10] == 0.0
    with pytest.raises(ValueError):
        co.absorption(co.Grid(4, 4, 4, LAM / 8, LAM, 1.0, (1, 1, 1), (1, 1, 1), corner="mean"))
