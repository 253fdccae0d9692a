"""Landau-Lifshitz-Gilbert time integration of a batch of islands, plain FP64
(oracle; test infrastructure).

The paper solves "the Landau-Lifshitz-Gilbert equation at 0 K" for the
recording simulations (Sec. II.A) with the head field moved over the island at
the head velocity and scaled with a rise time (Sec. II.A, II.C), plus a
globally applied constant field H_ext (Sec. II.C).  It does not print the
equation, the integrator or the switching criterion.  Readings used:

* LLG in Landau-Lifshitz form, Gilbert damping:
      dm/dt = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)],  B = mu0 H_eff (T),
  gamma = 1.76085963023e11 rad/(s T); no thermal field (0 K).
* effective field B = B_ex + B_an + B_d + ramp(t) (B_head + B_uniform) + B_ext,b
  with ramp(t) = min(1, t / t_rise); the head map is sampled at
  (x_i + pos_x - (x0 + v t), y_i + pos_y, z_i).
* per-island jitter scales Ms (exchange field 1/s, demag source s) and Ku
  (anisotropy field Ku_s / Ms_s); the easy axis u is per island.
* Heun predictor-corrector, |m| renormalised after BOTH the predictor and the
  corrector:
      k1 = f(m_n, t_n);  m* = N(m_n + h k1);  k2 = f(m*, t_n + h);
      m_{n+1} = N(m_n + h/2 (k1 + k2)),  N(v) = v / |v|.
* the output interval dt is split into k equal integrator steps h = dt / k
  (k from `stable_substeps`, chosen so that gamma' B_max h <= 0.5).
* switch detector: <m_z> = sum_i V_i m_z,i / sum_i V_i after every integrator
  step; the first step with <m_z> <= 0 gives t_sw by linear interpolation
  between the two steps; switched = <m_z>(t_end) <= 0; t_sw = -1 if no crossing.
"""
from __future__ import annotations

import math

import numpy as np

from .headfield import trilinear

GAMMA = 1.76085963023e11          # rad / (s T)
GAMMA_PS = GAMMA * 1e-12          # rad / (ps T)
MU0 = 4e-7 * math.pi

T_EXCHANGE, T_ANISOTROPY, T_DEMAG, T_HEAD, T_UNIFORM = 1, 2, 4, 8, 16


class Batch:
    """One batch of islands sharing one mesh (the oracle's view of a run)."""

    def __init__(self, ops, islands, params, head_map=None, demag=None):
        self.ops = ops
        self.p = params
        self.Ms_s = np.asarray(islands.Ms_scale, np.float64)
        self.Ku_s = np.asarray(islands.Ku_scale, np.float64)
        self.u = np.asarray(islands.u, np.float64)
        self.pos = np.asarray(islands.pos_nm, np.float64)
        self.Hext = np.asarray(islands.Hext_T, np.float64)
        self.map = head_map
        self.N = ops.demag if demag is None else demag
        self.B = self.Ms_s.shape[0]
        self.w = ops.V / ops.V.sum()

    # ---------------- effective field -----------------
    def ramp(self, t_ps: float) -> float:
        return 1.0 if self.p.rise_ps <= 0 else min(1.0, t_ps / self.p.rise_ps)

    def field(self, m: np.ndarray, t_ps: float, mask: int | None = None) -> np.ndarray:
        mask = self.p.term_mask if mask is None else mask
        ops, n = self.ops, self.ops.n
        B = np.zeros_like(m)
        if mask & T_EXCHANGE:
            B += -np.matmul(ops.S, m) / self.Ms_s[:, None, None]
        if mask & T_ANISOTROPY:
            coef = (2.0 * ops.Ku / ops.Ms)[None, :] * (self.Ku_s / self.Ms_s)[:, None]   # T
            mu = np.einsum("bic,bc->bi", m, self.u)
            B += (coef * mu)[:, :, None] * self.u[:, None, :]
        if mask & T_DEMAG:
            M = (ops.Ms[None, :, None] * self.Ms_s[:, None, None]) * m          # A/m
            Mp = M.transpose(0, 2, 1).reshape(self.B, 3 * n)                    # c*n + i
            H = -(Mp @ self.N.T)
            B += MU0 * H.reshape(self.B, 3, n).transpose(0, 2, 1)
        r = self.ramp(t_ps)
        if (mask & T_HEAD) and self.map is not None:
            xh = self.p.x0_nm + self.p.v_m_per_s * 1e-3 * t_ps
            pnt = np.empty((self.B, n, 3))
            pnt[:, :, 0] = ops.xyz[None, :, 0] + self.pos[:, None, 0] - xh
            pnt[:, :, 1] = ops.xyz[None, :, 1] + self.pos[:, None, 1]
            pnt[:, :, 2] = ops.xyz[None, :, 2]
            B += r * trilinear(self.map.B_T, self.map.origin_nm, self.map.h_nm, pnt)
        if mask & T_UNIFORM:
            B += r * np.asarray(self.p.uniform_T, np.float64)[None, None, :]
            B += self.Hext[:, None, :]
        return B

    def rhs(self, m: np.ndarray, t_ps: float) -> np.ndarray:
        gp = GAMMA_PS / (1.0 + self.p.alpha ** 2)
        Bf = self.field(m, t_ps)
        mxB = np.cross(m, Bf)
        return -gp * (mxB + self.p.alpha * np.cross(m, mxB))

    def mz_avg(self, m: np.ndarray) -> np.ndarray:
        return m[:, :, 2] @ self.w

    # ---------------- energy (J) for the damping check -----------------
    def energy(self, m: np.ndarray, t_ps: float) -> np.ndarray:
        ops, n, mask = self.ops, self.ops.n, self.p.term_mask
        Vm3 = ops.V * 1e-27
        E = np.zeros(self.B)
        if mask & T_EXCHANGE:
            E += np.einsum("bic,ij,bjc->b", m, ops.K_A, m) * 1e-9
        if mask & T_ANISOTROPY:
            mu = np.einsum("bic,bc->bi", m, self.u)
            E += -np.einsum("i,bi->b", Vm3 * ops.Ku, mu ** 2) * self.Ku_s
        Msn = ops.Ms[None, :] * self.Ms_s[:, None]
        if mask & T_DEMAG:
            M = Msn[:, :, None] * m
            Mp = M.transpose(0, 2, 1).reshape(self.B, 3 * n)
            NM = Mp @ self.N.T
            E += 0.5 * MU0 * np.einsum("bk,bk,k->b", Mp, NM, np.tile(Vm3, 3))
        zee = np.zeros_like(m)
        r = self.ramp(t_ps)
        if (mask & T_HEAD) and self.map is not None:
            zee += self.field(m, t_ps, T_HEAD)
        if mask & T_UNIFORM:
            zee += r * np.asarray(self.p.uniform_T, np.float64)[None, None, :] + self.Hext[:, None, :]
        E += -np.einsum("bi,bic,bic->b", Msn * Vm3[None, :], m, zee)
        return E

    # ---------------- integration -----------------
    def run(self, m0: np.ndarray | None = None, sample_every: int = 0, on_step=None):
        """Integrate from t0 to t_end; returns dict with m, switched, t_sw, mz,
        status, and samples (m after every `sample_every` output intervals)."""
        p = self.p
        n = self.ops.n
        k = int(p.substeps)
        h = p.dt_ps / k
        m = np.zeros((self.B, n, 3))
        m[:, :, 2] = 1.0
        if m0 is not None:
            m = np.array(m0, dtype=np.float64, copy=True)
        mz_prev = self.mz_avg(m)
        t_sw = np.where(mz_prev <= 0, p.t0_ps, -1.0)
        crossed = mz_prev <= 0
        samples = []
        n_int = p.n_intervals
        for it in range(n_int):
            for j in range(k):
                t_n = p.t0_ps + (it * k + j) * h
                k1 = self.rhs(m, t_n)
                ms = m + h * k1
                ms /= np.linalg.norm(ms, axis=2, keepdims=True)
                k2 = self.rhs(ms, t_n + h)
                mn = m + 0.5 * h * (k1 + k2)
                mn /= np.linalg.norm(mn, axis=2, keepdims=True)
                m = mn
                mz = self.mz_avg(m)
                new = (~crossed) & (mz <= 0)
                if np.any(new):
                    frac = mz_prev[new] / (mz_prev[new] - mz[new])
                    t_sw[new] = t_n + h * frac
                    crossed |= new
                mz_prev = mz
                if on_step is not None:
                    on_step(m, t_n + h)
            if sample_every and (it + 1) % sample_every == 0:
                samples.append(m.copy())
        status = np.where(np.all(np.isfinite(m), axis=(1, 2)), 0, 1).astype(np.int32)
        return dict(m=m, switched=mz_prev <= 0, t_sw=t_sw, mz=mz_prev, status=status,
                    samples=samples)


def field_bound(batch: Batch) -> float:
    """Upper bound of |B_eff| (T) used to pick the integrator step."""
    ops, p = batch.ops, batch.p
    lam = ops.exchange_lambda_max() / float(np.min(batch.Ms_s))
    an = float(np.max(2.0 * ops.Ku / ops.Ms) * np.max(batch.Ku_s / batch.Ms_s))
    dm = MU0 * float(np.max(ops.Ms) * np.max(batch.Ms_s))
    hd = float(np.max(np.linalg.norm(batch.map.B_T, axis=-1))) if batch.map is not None else 0.0
    un = float(np.linalg.norm(p.uniform_T)) + float(np.max(np.linalg.norm(batch.Hext, axis=1)))
    return lam + an + dm + hd + un


def stable_substeps(batch: Batch, courant: float = 0.5) -> int:
    """Smallest k with gamma/(1+alpha^2) * B_max * dt / k <= courant."""
    gp = GAMMA_PS / (1.0 + batch.p.alpha ** 2)
    return max(1, int(math.ceil(gp * field_bound(batch) * batch.p.dt_ps / courant)))
