"""Pins of the oracle's P1 FEM part against exact properties of linear
finite elements (independent of the oracle's own formulas)."""
import math

import numpy as np
import pytest

from oracle import fem
from paper_1603_09493_gb300 import synth


@pytest.fixture(scope="module")
def small():
    m = synth.small_island_mesh()
    ops = fem.MeshOperators(m.xyz_nm, m.tets, m.tet_region, synth.ecc_materials(), with_demag=False)
    return m, ops


def test_volume_is_polygon_prism(small):
    m, ops = small
    exact = synth.polygon_area_nm2(m) * m.height_nm
    assert abs(ops.vol.sum() - exact) < 1e-12 * exact
    assert abs(ops.V.sum() - exact) < 1e-12 * exact
    assert np.all(ops.vol > 0)


def test_gradients_reproduce_linear_functions(small):
    _, ops = small
    # sum_i grad(phi_i) = 0 and sum_i x_i[d] grad(phi_i) = e_d on every tet
    assert np.abs(ops.grads.sum(axis=1)).max() < 1e-12
    xt = ops.xyz[ops.tets]                                   # [nt][4][3]
    J = np.einsum("tkd,tke->tde", xt, ops.grads)
    assert np.abs(J - np.eye(3)[None]).max() < 1e-12


def test_stiffness_rows_sum_to_zero_and_symmetric(small):
    _, ops = small
    K = ops.K_A
    scale = np.abs(K).max()
    assert np.abs(K.sum(axis=1)).max() < 1e-13 * scale * K.shape[0]
    assert np.abs(K - K.T).max() < 1e-14 * scale


def test_linear_field_energy_is_exact(small):
    m, ops = small
    # f(x) = a.x + b has |grad f|^2 = |a|^2; P1 integrates it exactly: f K f = sum_t A_t vol_t |a|^2
    a = np.array([0.3, -0.7, 0.2])
    f = ops.xyz @ a + 1.5
    mats = synth.ecc_materials()
    A_t = mats[m.tet_region, 2]
    exact = float(np.sum(A_t * ops.vol)) * float(a @ a)
    assert abs(f @ ops.K_A @ f - exact) < 1e-12 * exact


def test_uniform_magnetisation_has_no_exchange_field(small):
    _, ops = small
    mm = np.zeros((2, ops.n, 3))
    mm[0, :, 2] = 1.0
    mm[1, :] = np.array([0.6, 0.0, 0.8])
    B = ops.exchange_field(mm, np.array([1.0, 1.1]))
    assert np.abs(B).max() < 1e-9 * np.abs(ops.S).max()


def test_spin_wave_exchange_field():
    # m = (sin kz, 0, cos kz) on a tall column: lap m = -k^2 m, so
    # B_ex = (2A/Ms) lap m = -(2A/Ms) k^2 m away from the ends (O(h^2) error of lumped P1)
    mesh = synth.layered_island_mesh(6.0, 20.0, 0.0001, rings=2, hard_slabs=40, soft_slabs=1,
                                     seed=3, perturb=0.0)
    mats = np.array([[1e6, 0.0, 1e-11]] * 3)
    ops = fem.MeshOperators(mesh.xyz_nm, mesh.tets, mesh.tet_region, mats, with_demag=False)
    k = 2 * math.pi / 10.0
    z = ops.xyz[:, 2]
    m = np.stack([np.sin(k * z), 0 * z, np.cos(k * z)], 1)[None]
    B = ops.exchange_field(m, np.ones(1))[0]
    inner = (z > 3.0) & (z < 17.0)
    pre = 2 * 1e-11 / 1e6 * 1e18 * k * k                   # T
    ratio = -np.einsum("ic,ic->i", B[inner], m[0, inner]) / pre
    assert np.all(np.abs(ratio - 1.0) < 0.03), (ratio.min(), ratio.max())
    # the field is parallel to m (no transverse part) for this mode
    perp = B[inner] + ratio[:, None] * pre * m[0, inner]
    assert np.abs(perp).max() < 0.03 * pre


def test_exchange_lambda_max_is_rayleigh_bound(small):
    _, ops = small
    lam = ops.exchange_lambda_max()
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.standard_normal(ops.n)
        d = ops.Ms * ops.V
        # generalised Rayleigh quotient of S = D^-1 K_A (2e18) is below lambda_max
        q = 2e18 * (x @ ops.K_A @ x) / (x @ (d * x))
        assert q <= lam * (1 + 1e-12)
    # Gershgorin bound from the other side
    gersh = np.max(np.sum(np.abs(ops.S), axis=1))
    assert lam <= gersh * (1 + 1e-12)
