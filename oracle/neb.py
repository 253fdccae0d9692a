"""Nudged elastic band for the energy barrier of an island in the head's fringing
field (Sec. II.C, adjacent-track erasure), plain FP64 (oracle; test
infrastructure).

The paper places the adjacent bit in the fringing field at the down-track
position of the lowest barrier, computes the switching barrier E_B with the
nudged elastic band method, and turns it into an error rate with Eq. (3):
tau = exp(E_B / kT) / f0, BER_adj = t_write / tau (f0 = 130 GHz, t_write = 1 ns,
T = 300 K).  It does not spell out the band.  Readings used (the standard
method of Henkelman and Jonsson, J. Chem. Phys. 113, 9978 (2000), with the
climbing image of Henkelman, Uberuaga and Jonsson, ibid. 9901, written for
unit vectors at every node):

* a band of P images m^0 .. m^{P-1} of the island, [n][3] unit vectors each;
  distances and inner products use the lumped volume weights w_i = V_i / sum V:
      <a, b> = sum_i w_i a_i . b_i,   |a| = sqrt(<a, a>);
* force density of an image: g_i = Ms_i B_i_perp (MA/m x T), with B the
  effective field of the image and B_perp = B - (B . m_i) m_i, the component in
  the tangent plane of m_i (minus the energy gradient in the weighted metric);
* tangent of an interior image k from its neighbours' energies (the improved
  tangent): t = m^{k+1} - m^k if E^{k+1} > E^k > E^{k-1};  t = m^k - m^{k-1} if
  E^{k+1} < E^k < E^{k-1}; otherwise the two differences weighted by
  dEmax = max(|E^{k+1} - E^k|, |E^{k-1} - E^k|) and dEmin = min(...), the larger
  weight on the side of the higher neighbour;  then projected onto the tangent
  plane of every m_i^k and normalised, |t| = 1;
* band force: g - <g, t> t + kappa (|m^{k+1} - m^k| - |m^k - m^{k-1}|) t;
  the climbing image (the interior image of highest energy, once climbing is on)
  takes g - 2 <g, t> t and no spring;
* the two end images relax by their own force g (they are minima of the field);
* every image moves at once (Jacobi): m_i <- N(m_i + step * force_i),
  N(v) = v / |v|;
* E_B = max over interior images of E - E^0 at the end.
"""
from __future__ import annotations

import math

import numpy as np

KB = 1.380649e-23          # J/K


def great_circle_path(n: int, P: int, axis: str = "x") -> np.ndarray:
    """Initial band: uniform states rotating from +z to -z through +axis."""
    th = np.linspace(0.0, math.pi, P)
    m = np.zeros((P, n, 3))
    c = {"x": 0, "y": 1}[axis]
    m[:, :, c] = np.sin(th)[:, None]
    m[:, :, 2] = np.cos(th)[:, None]
    return m


def _normalise(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _perp(v: np.ndarray, m: np.ndarray) -> np.ndarray:
    return v - np.sum(v * m, axis=-1, keepdims=True) * m


def _dot(a: np.ndarray, b: np.ndarray, w: np.ndarray) -> float:
    return float(np.sum(w[:, None] * a * b))


def tangent(m_prev, m, m_next, E_prev, E, E_next, w):
    """Improved tangent of an interior image, projected and normalised."""
    dp, dm = m_next - m, m - m_prev
    if E_next > E > E_prev:
        t = dp
    elif E_next < E < E_prev:
        t = dm
    else:
        dmax = max(abs(E_next - E), abs(E_prev - E))
        dmin = min(abs(E_next - E), abs(E_prev - E))
        t = dp * dmax + dm * dmin if E_next > E_prev else dp * dmin + dm * dmax
    t = _perp(t, m)
    return t / math.sqrt(_dot(t, t, w))


def neb(m_band, field_fn, energy_fn, msn, w, iters, step, spring, climb_after=-1):
    """Relax a band.

    m_band   [D][P][n][3] initial images of D independent bands
    field_fn m [D*P][n][3] -> effective field B (T), same shape
    energy_fn m [D*P][n][3] -> energy (J) [D*P]
    msn      [D][n] Ms_i of each band's island (MA/m)
    w        [n] volume weights (sum 1)
    Returns dict(m [D][P][n][3], E [D][P] at the final band, E_B [D] (J),
    force [D][P] max_i |band force_i| of the last iteration)."""
    m = np.array(m_band, np.float64)
    D, P, n, _ = m.shape
    force = np.zeros((D, P))
    for it in range(iters):
        flat = m.reshape(D * P, n, 3)
        B = field_fn(flat).reshape(D, P, n, 3)
        E = energy_fn(flat).reshape(D, P)
        new = np.empty_like(m)
        for d in range(D):
            ci = 1 + int(np.argmax(E[d, 1:P - 1])) if (climb_after >= 0 and it >= climb_after) else -1
            for k in range(P):
                g = msn[d][:, None] * _perp(B[d, k], m[d, k])
                if 0 < k < P - 1:
                    t = tangent(m[d, k - 1], m[d, k], m[d, k + 1], E[d, k - 1], E[d, k], E[d, k + 1], w)
                    s = _dot(g, t, w)
                    if k == ci:
                        f = g - 2.0 * s * t
                    else:
                        dn = math.sqrt(_dot(m[d, k + 1] - m[d, k], m[d, k + 1] - m[d, k], w))
                        dp = math.sqrt(_dot(m[d, k] - m[d, k - 1], m[d, k] - m[d, k - 1], w))
                        f = g - s * t + spring * (dn - dp) * t
                else:
                    f = g
                force[d, k] = float(np.max(np.linalg.norm(f, axis=-1)))
                new[d, k] = _normalise(m[d, k] + step * f)
        m = new
    E = energy_fn(m.reshape(D * P, n, 3)).reshape(D, P)
    return dict(m=m, E=E, E_B=E[:, 1:P - 1].max(axis=1) - E[:, 0], force=force)


def island_band(ops, islands, params, head_map, m_band, iters, step, spring, climb_after=-1):
    """The band for D islands of one mesh under the head field frozen at the head
    position params.x0_nm (ramp 1: params.rise_ps = 0, params.v_m_per_s = 0).
    islands: D islands; each band's images share its island's parameters."""
    from .llg import Batch
    D, P = m_band.shape[:2]
    rep = islands.subset(np.repeat(np.arange(D), P))
    batch = Batch(ops, rep, params, head_map=head_map)
    msn = (ops.Ms[None, :] * np.asarray(islands.Ms_scale, np.float64)[:, None]) * 1e-6
    w = ops.V / ops.V.sum()
    return neb(m_band, lambda m: batch.field(m, 0.0), lambda m: batch.energy(m, 0.0), msn, w, iters, step, spring,
               climb_after)


def barrier_kT(E_B_J, T_K: float = 300.0):
    return np.asarray(E_B_J) / (KB * T_K)
