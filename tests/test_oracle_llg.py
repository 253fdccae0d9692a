"""Pins of the oracle's LLG integrator, fields and switch detector against
closed forms: Larmor precession, the damped reversal time of a single spin in
an antiparallel field, the Stoner-Wohlfarth astroid, the linear modes of a
meshed two-layer island (an eigenproblem of its exchange and anisotropy
operators), trilinear exactness on affine fields, energy decay under damping,
and |m| = 1."""
import math

import numpy as np
import pytest

from oracle import fem, headfield, llg
from paper_1603_09493_gb300 import synth

HARD = np.array([[0.8e6, 0.9e6, 1e-11]] * 3)


def _one_tet_ops(mats=HARD):
    xyz = np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    tets = np.array([[0, 1, 2, 3]])
    return fem.MeshOperators(xyz, tets, np.array([0]), mats, with_demag=False)


def _tilted(n, B, theta):
    m = np.zeros((B, n, 3))
    m[:, :, 0] = math.sin(theta)
    m[:, :, 2] = math.cos(theta)
    return m


def test_larmor_precession():
    ops = _one_tet_ops()
    B0 = 1.0
    p = synth.RunParams(dt_ps=0.1, substeps=10, t_end_ps=100.0, alpha=0.0, rise_ps=0.0,
                        uniform_T=(0.0, 0.0, B0), term_mask=synth.TERM_UNIFORM)
    b = llg.Batch(ops, synth.nominal_islands(1), p)
    th = math.radians(30)
    r = b.run(_tilted(4, 1, th))
    m = r["m"][0, 0]
    phase = math.atan2(m[1], m[0])
    expect = (llg.GAMMA_PS * B0 * p.t_end_ps) % (2 * math.pi)
    expect = (expect + math.pi) % (2 * math.pi) - math.pi
    assert abs(phase - expect) < 1e-4
    # Heun + renormalisation shortens the step vector by O((omega h)^4) per step:
    # m_z drifts by at most N (omega h)^4 / 8 ~ 1.2e-8 here
    assert abs(m[2] - math.cos(th)) < 1.2e-8
    # 28.025 GHz/T
    assert abs(llg.GAMMA / (2 * math.pi) / 1e9 - 28.0249514) < 1e-6


def test_damped_reversal_time_closed_form():
    # field B along -z, no anisotropy: tan(theta/2) = tan(theta0/2) exp(-gamma' alpha B t),
    # theta measured from -z; <m_z> = 0 when theta = pi/2
    ops = _one_tet_ops()
    B0, alpha, delta = 1.0, 0.1, 0.1
    p = synth.RunParams(dt_ps=0.1, substeps=2, t_end_ps=300.0, alpha=alpha, rise_ps=0.0,
                        uniform_T=(0.0, 0.0, -B0), term_mask=synth.TERM_UNIFORM)
    b = llg.Batch(ops, synth.nominal_islands(1), p)
    r = b.run(_tilted(4, 1, delta))
    gp = llg.GAMMA_PS / (1 + alpha ** 2)
    t_star = math.log(1.0 / math.tan(delta / 2)) / (gp * alpha * B0)
    assert r["switched"][0]
    assert abs(r["t_sw"][0] - t_star) < 0.05, (r["t_sw"][0], t_star)
    th_end = 2 * math.atan(math.tan((math.pi - delta) / 2) * math.exp(-gp * alpha * B0 * p.t_end_ps))
    assert abs(r["mz"][0] + math.cos(th_end)) < 1e-4, (r["mz"][0], -math.cos(th_end))


def _sw_threshold(psi_deg, hs):
    ops = _one_tet_ops()
    HK = 2 * 0.9e6 / 0.8e6                                   # mu0 H_K in tesla
    psi = math.radians(psi_deg)
    isl = synth.nominal_islands(len(hs))
    isl.Hext_T[:] = np.stack([np.sin(psi) * hs * HK, 0 * hs, -np.cos(psi) * hs * HK], 1)
    p = synth.RunParams(dt_ps=0.5, substeps=4, t_end_ps=1500.0, alpha=1.0, rise_ps=0.0,
                        term_mask=synth.TERM_ANISOTROPY | synth.TERM_UNIFORM)
    r = llg.Batch(ops, isl, p).run()
    sw = r["switched"]
    assert not sw[0] and sw[-1]
    first = int(np.argmax(sw))
    assert np.all(sw[first:])
    return hs[first - 1], hs[first]


@pytest.mark.parametrize("psi_deg", [10.0, 45.0])
def test_stoner_wohlfarth_astroid(psi_deg):
    psi = math.radians(psi_deg)
    h_sw = (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** -1.5
    if psi_deg == 10.0:
        assert abs(h_sw - 0.6738) < 1e-4
    if psi_deg == 45.0:
        assert abs(h_sw - 0.5) < 1e-12
    hs = h_sw * np.linspace(0.97, 1.03, 25)
    lo, hi = _sw_threshold(psi_deg, hs)
    assert lo <= h_sw * 1.01 and hi >= h_sw * 0.99, (lo, hi, h_sw)
    assert abs(0.5 * (lo + hi) / h_sw - 1.0) < 0.01


def test_trilinear_is_exact_for_affine_fields_and_clamps():
    nz, ny, nx = 5, 6, 7
    h = 0.7
    origin = np.array([-2.0, 1.0, 0.5])
    zs, ys, xs = (origin[2] + h * np.arange(nz), origin[1] + h * np.arange(ny),
                  origin[0] + h * np.arange(nx))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [-0.1, 0.2, 0.25]])
    c0 = np.array([0.1, -0.2, 0.3])
    pts = np.stack([X, Y, Z], -1)
    B = pts @ A.T + c0
    rng = np.random.default_rng(2)
    lo, hi = origin, origin + h * (np.array([nx, ny, nz]) - 1)
    q = lo + rng.random((200, 3)) * (hi - lo)
    out = headfield.trilinear(B, origin, h, q)
    assert np.abs(out - (q @ A.T + c0)).max() < 1e-12
    # outside the box: value of the nearest point of the box
    far = np.array([[hi[0] + 5.0, q[0, 1], q[0, 2]], [lo[0] - 3.0, lo[1] - 1.0, hi[2] + 2.0]])
    clamped = np.clip(far, lo, hi)
    assert np.abs(headfield.trilinear(B, origin, h, far) - (clamped @ A.T + c0)).max() < 1e-12


def test_head_field_moves_with_head():
    hm = synth.synthetic_head_map()
    # a node at the head centre line sees the peak direction; the value moves at v
    mesh = synth.small_island_mesh()
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, synth.ecc_materials(),
                            with_demag=False)
    p = synth.RunParams(rise_ps=0.0, v_m_per_s=20.0, x0_nm=-10.0, use_map=True,
                        term_mask=synth.TERM_HEAD)
    b = llg.Batch(ops, synth.nominal_islands(1), p, head_map=hm)
    m = _tilted(ops.n, 1, 0.0)
    B500 = b.field(m, 500.0)                  # head centre over x = 0
    B0 = b.field(m, 0.0)
    centre = np.argmin(np.linalg.norm(ops.xyz[:, :2], axis=1) + np.abs(ops.xyz[:, 2] - 10.0))
    assert np.linalg.norm(B500[0, centre]) > np.linalg.norm(B0[0, centre]) * 1.5
    d = B500[0, centre] / np.linalg.norm(B500[0, centre])
    assert abs(d[1] - math.sin(math.radians(25))) < 1e-6 and d[2] < 0


@pytest.fixture(scope="module")
def small_ops():
    m = synth.small_island_mesh()
    return fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials())


def test_energy_decays_and_norm_is_kept(small_ops):
    ops = small_ops
    W = np.tile(ops.V, 3)
    Nsym = 0.5 * (ops.demag + (ops.demag.T * W[None, :]) / W[:, None])
    isl = synth.jittered_islands(3, seed=5)
    p = synth.RunParams(dt_ps=0.1, t_end_ps=20.0, alpha=0.5, rise_ps=0.0,
                        uniform_T=synth.uniform_field(0.8, 150.0),
                        term_mask=synth.TERM_EXCHANGE | synth.TERM_ANISOTROPY | synth.TERM_DEMAG | synth.TERM_UNIFORM)
    b = llg.Batch(ops, isl, p, demag=Nsym)
    p.substeps = llg.stable_substeps(b)
    x = ops.xyz
    m0 = np.stack([0.3 * np.sin(x[:, 0]), 0.2 * np.cos(x[:, 1]), np.ones(ops.n)], 1)
    m0 = np.broadcast_to(m0 / np.linalg.norm(m0, axis=1, keepdims=True), (3, ops.n, 3)).copy()
    energies, norms = [b.energy(m0, 0.0)], []

    def on_step(m, t):
        energies.append(b.energy(m, t))
        norms.append(np.abs(np.linalg.norm(m, axis=2) - 1.0).max())

    b.run(m0, on_step=on_step)
    E = np.array(energies)
    dE = np.diff(E, axis=0)
    assert np.all(dE <= 1e-9 * np.abs(E[:-1])), dE.max()
    assert E[-1].max() < E[0].min()
    assert max(norms) < 1e-14


@pytest.mark.parametrize("alpha", [0.0, 0.1])
def test_linear_modes_of_a_meshed_island(alpha):
    # Small deviations from the uniform state m = z of the two-layer island, under a uniform field
    # B0 along the easy axis z, demag off. To first order in w = m_x + i m_y the LLG becomes
    #   dw/dt = gamma' (i - alpha) A w,  A = diag(B0 + 2 Ku_i / Ms_i) + S,
    # with S the lumped exchange operator (B_ex = -S m, zero row sums, so the exchange field of
    # the uniform state vanishes). A is a diagonal scaling of a symmetric matrix, so its
    # eigenvalues lam are real: each mode precesses at gamma' lam and decays at gamma' alpha lam.
    # Heun on a linear system is the map w -> (1 + z + z^2/2) w, z = h gamma' (i - alpha) A.
    m = synth.small_island_mesh()
    ops = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials(), with_demag=False)
    n, B0 = ops.n, 0.5
    A = np.diag(B0 + 2.0 * ops.Ku / ops.Ms) + ops.S
    lam, V = np.linalg.eig(A)
    assert np.abs(lam.imag).max() == 0.0 and lam.real.min() > B0
    lam, V = lam.real, V.real
    p = synth.RunParams(dt_ps=0.1, t_end_ps=5.0, alpha=alpha, rise_ps=0.0, uniform_T=(0.0, 0.0, B0),
                        term_mask=synth.TERM_EXCHANGE | synth.TERM_ANISOTROPY | synth.TERM_UNIFORM)
    b = llg.Batch(ops, synth.nominal_islands(1), p)
    p.substeps = llg.stable_substeps(b)
    h, steps = p.dt_ps / p.substeps, p.n_intervals * p.substeps
    gp = llg.GAMMA_PS / (1 + alpha ** 2)

    def start(w):
        m0 = np.zeros((1, n, 3))
        m0[0, :, 0], m0[0, :, 1], m0[0, :, 2] = w.real, w.imag, 1.0
        return m0 / np.linalg.norm(m0, axis=2, keepdims=True)

    # every mode at once, against the discrete linear map: a deviation of 1e-5 leaves
    # nonlinear terms of relative size 1e-10
    m0 = start(1e-5 * np.random.default_rng(3).standard_normal(n).astype(complex))
    w0 = m0[0, :, 0] + 1j * m0[0, :, 1]
    r = b.run(m0)
    w = r["m"][0, :, 0] + 1j * r["m"][0, :, 1]
    z = h * gp * (1j - alpha) * lam
    w_lin = V @ ((1 + z + z * z / 2) ** steps * np.linalg.solve(V, w0))
    assert np.abs(w - w_lin).max() < 1e-6 * np.abs(w_lin).max()
    # the lowest mode alone, against the continuous solution: Heun's phase error per step is
    # (omega h)^3 / 6, and its amplitude error is of the same order
    v = V[:, np.argmin(lam)]
    m0 = start(1e-5 * v / np.abs(v).max() + 0j)
    r = b.run(m0)
    w = r["m"][0, :, 0] + 1j * r["m"][0, :, 1]
    om = gp * lam.min()
    w_ex = (m0[0, :, 0] + 1j * m0[0, :, 1]) * np.exp((1j - alpha) * om * p.t_end_ps)
    bound = steps * ((om * h) ** 3 / 6) * math.hypot(1.0, alpha) ** 3
    assert np.abs(w - w_ex).max() < 2.0 * bound * np.abs(w_ex).max() + 1e-9 * np.abs(w_ex).max()


def test_stable_substeps_scales_with_dt(small_ops):
    isl = synth.nominal_islands(1)
    p1 = synth.RunParams(dt_ps=0.1)
    p2 = synth.RunParams(dt_ps=0.4)
    k1 = llg.stable_substeps(llg.Batch(small_ops, isl, p1))
    k2 = llg.stable_substeps(llg.Batch(small_ops, isl, p2))
    assert k1 >= 2 and 4 * k1 - 4 <= k2 <= 4 * k1


def test_small_island_switching_converges_in_step(small_ops):
    # self-consistency, not a pin: halving the integrator step moves t_sw by < 0.5 ps
    p = synth.RunParams(dt_ps=0.1, t_end_ps=120.0, alpha=0.1, rise_ps=50.0,
                        uniform_T=synth.uniform_field(1.2, 170.0))
    b = llg.Batch(small_ops, synth.nominal_islands(1), p)
    k = llg.stable_substeps(b)
    p.substeps = k
    r1 = b.run()
    p.substeps = 2 * k
    r2 = b.run()
    assert r1["switched"][0] and r2["switched"][0]
    assert abs(r1["t_sw"][0] - r2["t_sw"][0]) < 0.5
