"""Thin Python layer over the C ABI: same operations, numpy/torch arguments.

Every computation runs in libbpmllg.so; these classes only own handles and
convert arguments.  Host arrays are numpy; device arrays are torch CUDA
tensors on the context's GPU, contiguous, of the dtype and extents each call
states (checked here: the library trusts a device pointer with the extents its
other arguments imply).
"""
from __future__ import annotations

import contextlib
import ctypes
from ctypes import byref, c_double, c_int32, c_void_p

import numpy as np

from . import _lib as L


def device_tensor(t, device: int, dtype: str, shape, name: str):
    """Check a tensor whose address goes to the library as a device pointer: a CUDA tensor on
    the context's device, of torch dtype `dtype` (a name, e.g. "float32"), contiguous, with the
    given extents (None: any).  Raises ValueError otherwise; returns t."""
    import torch
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: expected a torch CUDA tensor, got {type(t).__name__}")
    if t.device.index != device:
        raise ValueError(f"{name}: on cuda:{t.device.index}, the context is on cuda:{device}")
    if t.dtype != getattr(torch, dtype):
        raise ValueError(f"{name}: dtype {t.dtype}, expected torch.{dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    got = tuple(int(e) for e in t.shape)
    if len(got) != len(shape) or any(s is not None and e != int(s) for e, s in zip(got, shape)):
        want = tuple("*" if s is None else int(s) for s in shape)
        raise ValueError(f"{name}: shape {got}, expected {want}")
    return t


def run_params(p, precision: int = L.PREC_BF16X3, map_id: int = -1) -> L.bpm_run_params:
    """bpm_run_params from a synth.RunParams-like object."""
    q = L.bpm_run_params()
    q.dt_ps = p.dt_ps
    q.substeps = int(p.substeps)
    q.precision = int(precision)
    q.t0_ps = p.t0_ps
    q.alpha = p.alpha
    q.rise_ps = p.rise_ps
    q.v_m_per_s = p.v_m_per_s
    q.x0_nm = p.x0_nm
    q.map_id = int(map_id if getattr(p, "use_map", True) else -1)
    q.term_mask = int(p.term_mask)
    for c in range(3):
        q.uniform_T[c] = float(p.uniform_T[c])
    return q


def island_array(isl) -> np.ndarray:
    """Pack a synth.Islands into the C struct layout (bpm_island[B])."""
    B = len(isl)
    a = np.zeros(B, dtype=L.ISLAND_DTYPE)
    a["mesh_id"] = isl.mesh_id
    a["Ms_scale"] = isl.Ms_scale
    a["Ku_scale"] = isl.Ku_scale
    a["u"] = isl.u
    a["pos_nm"] = isl.pos_nm
    a["Hext_T"] = isl.Hext_T
    return a


class Context:
    def __init__(self, device: int = 0, stream=None):
        self.lib = L.load()
        h = c_void_p()
        s = None if stream is None else c_void_p(int(getattr(stream, "cuda_stream", stream)))
        L.check(self.lib.bpm_create(byref(h), int(device), s))
        self.h = h
        self.device = int(device)
        sp = c_void_p()
        L.check(self.lib.bpm_context_stream(h, byref(sp)))
        self.stream_ptr = int(sp.value or 0)

    @contextlib.contextmanager
    def device_order(self):
        """Order a library call that reads or writes torch device tensors against
        torch's current stream: the context stream waits for the work already
        queued on torch's stream (the producers of the inputs, and earlier users
        of memory the caching allocator hands out again), and torch's stream
        waits for the call's work before anything queued after it (readers of
        the outputs, frees of the inputs)."""
        import torch
        cur = torch.cuda.current_stream(self.device)
        if int(cur.cuda_stream) == self.stream_ptr:
            yield
            return
        ctx_stream = torch.cuda.ExternalStream(self.stream_ptr, device=torch.device("cuda", self.device))
        ctx_stream.wait_stream(cur)
        try:
            yield
        finally:
            cur.wait_stream(ctx_stream)

    def stable_substeps(self, islands, params, map_id: int = -1):
        """(k, field bound in T) of a run of these islands (bpm_stable_substeps): the
        library's integrator step count, the one a run with substeps = 0 takes."""
        isl = island_array(islands)
        q = run_params(params, L.PREC_FP32, map_id)
        k = c_int32()
        b = c_double()
        L.check(self.lib.bpm_stable_substeps(self.h, L.ptr(isl), len(isl), byref(q), byref(k), byref(b)))
        return k.value, b.value

    def close(self):
        if self.h:
            self.lib.bpm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- meshes
    def mesh_upload(self, mesh, mats, keep_f64: bool = False) -> int:
        xyz = np.ascontiguousarray(mesh.xyz_nm, np.float64)
        tets = np.ascontiguousarray(mesh.tets, np.int32)
        reg = np.ascontiguousarray(mesh.tet_region, np.int32)
        mats = np.asarray(mats, np.float64)
        if xyz.ndim != 2 or xyz.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4 or \
                reg.shape != (tets.shape[0],) or mats.ndim != 2:
            raise ValueError(f"mesh: xyz {xyz.shape} (n, 3), tets {tets.shape} (m, 4), regions {reg.shape} (m,), "
                             f"materials {mats.shape} (regions, fields)")
        cm = (L.bpm_region_mat * len(mats))(*[L.bpm_region_mat(*map(float, r)) for r in mats])
        mid = c_int32()
        L.check(self.lib.bpm_mesh_upload(self.h, L.ptr(xyz), xyz.shape[0], L.ptr(tets), tets.shape[0],
                                         L.ptr(reg), ctypes.cast(cm, c_void_p), len(mats),
                                         L.MESH_KEEP_F64 if keep_f64 else 0, byref(mid)))
        return mid.value

    def mesh_info(self, mesh_id: int) -> dict:
        info = L.bpm_mesh_info()
        L.check(self.lib.bpm_mesh_info_get(self.h, mesh_id, byref(info)))
        return {f: getattr(info, f) for f, _ in L.bpm_mesh_info._fields_ if f != "pad_"}

    def get_operator(self, mesh_id: int, which: int) -> np.ndarray:
        n = self.mesh_info(mesh_id)["n_nodes"]
        shape, dt = {L.OP_EXCHANGE_F32: ((n, n), np.float32), L.OP_DEMAG_F64: ((3 * n, 3 * n), np.float64),
                     L.OP_DEMAG_F32: ((3 * n, 3 * n), np.float32), L.OP_VOLUMES_F64: ((n,), np.float64),
                     L.OP_NODAL_MS_F64: ((n,), np.float64), L.OP_NODAL_KU_F64: ((n,), np.float64)}[which]
        out = np.zeros(shape, dt)
        L.check(self.lib.bpm_mesh_get_operator(self.h, mesh_id, which, L.ptr(out)))
        return out

    def mesh_release(self, mesh_id: int):
        """Free a mesh's device operators (bpm_mesh_release); no live batch may use it."""
        L.check(self.lib.bpm_mesh_release(self.h, int(mesh_id)))

    def headmap_release(self, map_id: int):
        """Free a head map (bpm_headmap_release); no live batch may use it."""
        L.check(self.lib.bpm_headmap_release(self.h, int(map_id)))

    def headmap_upload(self, hm) -> int:
        B = np.ascontiguousarray(hm.B_T, np.float32)
        org = np.ascontiguousarray(hm.origin_nm, np.float32)
        if B.ndim != 4 or B.shape[3] != 3 or org.shape != (3,):
            raise ValueError(f"head map: B_T {B.shape}, expected (nz, ny, nx, 3); origin {org.shape}, expected (3,)")
        nz, ny, nx = B.shape[:3]
        mid = c_int32()
        L.check(self.lib.bpm_headmap_upload(self.h, L.ptr(B), nx, ny, nz, float(hm.h_nm), L.ptr(org),
                                            byref(mid)))
        return mid.value

    def head_field(self, geometry, nx: int, ny: int, nz: int, h_nm: float, origin_nm, out=None):
        """Field of a saturated main pole on a voxel grid (bpm_head_field_solve).  geometry: a
        mapping with the bpm_pole_geometry field names.  Returns a synth.HeadMap (host), or fills
        the torch device tensor `out` ([nz][ny][nx][3] float32) and returns it."""
        from . import synth
        g = L.bpm_pole_geometry()
        for f, _ in L.bpm_pole_geometry._fields_:
            setattr(g, f, type(getattr(g, f))(geometry.get(f, 0)))
        org = np.ascontiguousarray(origin_nm, np.float32)
        if org.shape != (3,):
            raise ValueError(f"origin_nm: {org.shape[0] if org.ndim == 1 else org.shape} values, expected 3")
        if out is not None:
            device_tensor(out, self.device, "float32", (nz, ny, nx, 3), "out")
            with self.device_order():
                L.check(self.lib.bpm_head_field_solve(self.h, byref(g), int(nx), int(ny), int(nz), float(h_nm),
                                                      L.ptr(org), L.ptr(out), 1))
            return out
        B = np.zeros((nz, ny, nx, 3), np.float32)
        L.check(self.lib.bpm_head_field_solve(self.h, byref(g), int(nx), int(ny), int(nz), float(h_nm), L.ptr(org),
                                              L.ptr(B), 0))
        return synth.HeadMap(B_T=B, origin_nm=org.copy(), h_nm=float(h_nm), info=dict(geometry))

    # ---- batches
    def batch(self, islands, params, precision=L.PREC_BF16X3, map_id=-1) -> "Batch":
        return Batch(self, islands, params, precision, map_id)

    def run_batch(self, islands, params, n_intervals, precision=L.PREC_BF16X3, map_id=-1):
        isl = island_array(islands)
        q = run_params(params, precision, map_id)
        n = max(self.mesh_info(int(mid))["n_nodes"] for mid in np.unique(isl["mesh_id"]))
        B = len(isl)
        m = np.zeros((B, 3, n), np.float32)
        sw = np.zeros(B, np.uint8)
        tsw = np.zeros(B, np.float32)
        st = np.zeros(B, np.int32)
        L.check(self.lib.bpm_run_batch(self.h, L.ptr(isl), B, byref(q), int(n_intervals), L.ptr(m), n,
                                       L.ptr(sw), L.ptr(tsw), L.ptr(st)))
        return dict(m=m, switched=sw.astype(bool), t_sw=tsw, status=st)

    def run_batch_dev(self, islands, params, n_intervals, precision=L.PREC_BF16X3, map_id=-1):
        """bpm_run_batch with the results in torch device tensors on the context's device."""
        import torch
        isl = island_array(islands)
        q = run_params(params, precision, map_id)
        n = max(self.mesh_info(int(mid))["n_nodes"] for mid in np.unique(isl["mesh_id"]))
        B = len(isl)
        dev = torch.device("cuda", self.device)
        m = torch.empty((B, 3, n), dtype=torch.float32, device=dev)
        sw = torch.empty(B, dtype=torch.uint8, device=dev)
        tsw = torch.empty(B, dtype=torch.float32, device=dev)
        st = torch.empty(B, dtype=torch.int32, device=dev)
        with self.device_order():
            L.check(self.lib.bpm_run_batch_dev(self.h, L.ptr(isl), B, byref(q), int(n_intervals), L.ptr(m), n,
                                               L.ptr(sw), L.ptr(tsw), L.ptr(st)))
        return dict(m=m, switched=sw.bool(), t_sw=tsw, status=st)

    def run_plain(self, islands, params, n_intervals, map_id=-1):
        """One island per launch, FP32 GEMV demag (bpm_run_plain); returns results and device ms."""
        isl = island_array(islands)
        q = run_params(params, L.PREC_FP32, map_id)
        n = max(self.mesh_info(int(mid))["n_nodes"] for mid in np.unique(isl["mesh_id"]))
        B = len(isl)
        m = np.zeros((B, 3, n), np.float32)
        sw = np.zeros(B, np.uint8)
        tsw = np.zeros(B, np.float32)
        st = np.zeros(B, np.int32)
        ms = c_double()
        L.check(self.lib.bpm_run_plain(self.h, L.ptr(isl), B, byref(q), int(n_intervals), L.ptr(m), n, L.ptr(sw),
                                       L.ptr(tsw), L.ptr(st), byref(ms)))
        return dict(m=m, switched=sw.astype(bool), t_sw=tsw, status=st, device_ms=ms.value)

    def run_plain_f64(self, islands, params, n_intervals, map_id=-1):
        """One island per launch with every step in FP64 (bpm_run_plain_f64; the meshes
        must be uploaded with keep_f64=True); returns results (m float64) and device ms."""
        isl = island_array(islands)
        q = run_params(params, L.PREC_FP32, map_id)
        n = max(self.mesh_info(int(mid))["n_nodes"] for mid in np.unique(isl["mesh_id"]))
        B = len(isl)
        m = np.zeros((B, 3, n), np.float64)
        sw = np.zeros(B, np.uint8)
        tsw = np.zeros(B, np.float64)
        st = np.zeros(B, np.int32)
        ms = c_double()
        L.check(self.lib.bpm_run_plain_f64(self.h, L.ptr(isl), B, byref(q), int(n_intervals), L.ptr(m), n,
                                           L.ptr(sw), L.ptr(tsw), L.ptr(st), byref(ms)))
        return dict(m=m, switched=sw.astype(bool), t_sw=tsw, status=st, device_ms=ms.value)

    def llg_advance_noalloc(self, islands, params, n_intervals, m_dev, mz_dev=None, map_id=-1):
        """FP32 advance with no device allocation (bpm_llg_advance_noalloc):
        m_dev is a device tensor [B][3][ld] updated in place, ordered against
        torch's current stream."""
        isl = island_array(islands)
        q = run_params(params, L.PREC_FP32, map_id)
        device_tensor(m_dev, self.device, "float32", (len(isl), 3, None), "m_dev")
        if mz_dev is not None:
            device_tensor(mz_dev, self.device, "float32", (len(isl),), "mz_dev")
        with self.device_order():
            L.check(self.lib.bpm_llg_advance_noalloc(self.h, L.ptr(isl), len(isl), byref(q), int(n_intervals),
                                                     L.ptr(m_dev), int(m_dev.shape[-1]), L.ptr(mz_dev)))

    def neb(self, islands, n_images: int, max_iters: int, step: float, spring: float, climb_after: int = -1,
            precision: int = L.PREC_BF16X3, map_id: int = -1, head_x_nm: float = 0.0, uniform_T=(0.0, 0.0, 0.0),
            term_mask: int = L.TERM_ALL, m_init=None, force_tol: float = 0.0, check_every: int = 50,
            want_path: bool = False) -> dict:
        """Nudged elastic band of one band per island (bpm_neb_run); returns
        E [D][P] (J), E_B [D] (J), iters, max_force and, with want_path, m [D][P][3][n]."""
        isl = island_array(islands)
        D = len(isl)
        n = self.mesh_info(int(isl["mesh_id"][0]))["n_nodes"]
        q = L.bpm_neb_params(int(n_images), int(max_iters), int(climb_after), int(precision), int(map_id),
                             int(term_mask), int(check_every), 0, float(step), float(spring), float(force_tol),
                             float(head_x_nm), (c_double * 3)(*[float(x) for x in uniform_T]))
        E = np.zeros((D, n_images), np.float64)
        EB = np.zeros(D, np.float64)
        mi = None if m_init is None else np.ascontiguousarray(m_init, np.float32)
        if mi is not None and mi.shape != (D, int(n_images), 3, n):
            raise ValueError(f"m_init: shape {mi.shape}, expected ({D}, {int(n_images)}, 3, {n})")
        mp = np.zeros((D, n_images, 3, n), np.float32) if want_path else None
        it = c_int32()
        fm = c_double()
        L.check(self.lib.bpm_neb_run(self.h, L.ptr(isl), D, byref(q), L.ptr(mi), n, L.ptr(E), L.ptr(EB), L.ptr(mp),
                                     byref(it), byref(fm)))
        out = dict(E=E, E_B=EB, iters=it.value, max_force=fm.value)
        if want_path:
            out["m"] = mp
        return out

    def surrogate(self, sizes, params) -> "Surrogate":
        return Surrogate(self, sizes, params)


class Surrogate:
    """Handle of a device-resident MLP surrogate (bpm_surrogate_*)."""

    def __init__(self, ctx: Context, sizes, params):
        n_in, width, depth, n_out = sizes
        self.ctx, self.lib = ctx, ctx.lib
        self.n_in, self.n_out = n_in, n_out
        cfg = L.bpm_mlp_cfg(n_in, width, depth, n_out)
        flat = np.ascontiguousarray(params, np.float32).reshape(-1)
        widths = [int(n_in)] + [int(width)] * int(depth) + [int(n_out)]
        count = sum(a * b + b for a, b in zip(widths[:-1], widths[1:]))   # W [out][in], then b, per layer
        if flat.size != count:
            raise ValueError(f"expected {count} parameters for sizes {tuple(sizes)}, got {flat.size}")
        sid = c_int32()
        L.check(self.lib.bpm_surrogate_create(ctx.h, byref(cfg), L.ptr(flat), byref(sid)))
        self.sid = sid.value
        cnt = ctypes.c_int64()
        L.check(self.lib.bpm_surrogate_param_count(ctx.h, self.sid, byref(cnt)))
        self.P = cnt.value
        if flat.size != self.P:
            raise ValueError(f"expected {self.P} parameters, got {flat.size}")

    def params(self) -> np.ndarray:
        out = np.zeros(self.P, np.float32)
        L.check(self.lib.bpm_surrogate_get_params(self.ctx.h, self.sid, L.ptr(out)))
        return out

    def _host_rows(self, X, cols=None, name="X"):
        """Host rows [N][cols] (cols = n_in by default) as contiguous float32."""
        X = np.ascontiguousarray(X, np.float32)
        cols = self.n_in if cols is None else cols
        if X.ndim != 2 or X.shape[1] != cols:
            raise ValueError(f"{name}: shape {X.shape}, expected (N, {cols})")
        return X

    def _host_pairs(self, X, Y):
        X = self._host_rows(X)
        Y = self._host_rows(Y, self.n_out, "Y")
        if Y.shape[0] != X.shape[0]:
            raise ValueError(f"{X.shape[0]} inputs, {Y.shape[0]} labels")
        return X, Y

    def grad(self, X, Y):
        X, Y = self._host_pairs(X, Y)
        g = np.zeros(self.P, np.float32)
        loss = ctypes.c_float()
        L.check(self.lib.bpm_surrogate_grad(self.ctx.h, self.sid, L.ptr(X), L.ptr(Y), X.shape[0], L.ptr(g),
                                            byref(loss)))
        return g, loss.value

    def train(self, X, Y, epochs, batch, lr, weight_decay, beta1=0.9, beta2=0.999, eps=1e-8):
        X, Y = self._host_pairs(X, Y)
        cfg = L.bpm_train_cfg(int(epochs), int(batch), lr, weight_decay, beta1, beta2, eps, 0)
        steps = int(epochs) * ((X.shape[0] + int(batch) - 1) // int(batch))
        curve = np.zeros(steps, np.float32)
        L.check(self.lib.bpm_surrogate_train(self.ctx.h, self.sid, L.ptr(X), L.ptr(Y), X.shape[0], byref(cfg),
                                             L.ptr(curve)))
        return curve

    def infer(self, X) -> np.ndarray:
        on_dev = int(getattr(X, "is_cuda", False))
        if on_dev:
            import torch
            device_tensor(X, self.ctx.device, "float32", (None, self.n_in), "X")
            P = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        else:
            X = self._host_rows(X)
            P = np.zeros((X.shape[0], self.n_out), np.float32)
        with self.ctx.device_order() if on_dev else contextlib.nullcontext():
            L.check(self.lib.bpm_surrogate_infer(self.ctx.h, self.sid, L.ptr(X), X.shape[0], L.ptr(P), on_dev))
        return P

    def screen(self, X, n_designs: int, n_jitter: int):
        """Screened error rates per design [n_designs][n_out] (float64) from the
        design-major jitter samples X [n_designs * n_jitter][n_in]: column 0 the
        mean probability that the target island does not switch, the others the
        mean probability of their event (bpm_surrogate_screen)."""
        n_designs, n_jitter = int(n_designs), int(n_jitter)
        if X.shape[0] != n_designs * n_jitter:
            raise ValueError(f"{X.shape[0]} rows for {n_designs} designs x {n_jitter} jitter samples")
        on_dev = int(getattr(X, "is_cuda", False))
        if on_dev:
            import torch
            device_tensor(X, self.ctx.device, "float32", (n_designs * n_jitter, self.n_in), "X")
            R = torch.empty((n_designs, self.n_out), dtype=torch.float64, device=X.device)
        else:
            X = self._host_rows(X)
            R = np.zeros((n_designs, self.n_out), np.float64)
        with self.ctx.device_order() if on_dev else contextlib.nullcontext():
            L.check(self.lib.bpm_surrogate_screen(self.ctx.h, self.sid, L.ptr(X), n_designs, n_jitter, L.ptr(R),
                                                  on_dev))
        return R

    def save(self, path: str):
        L.check(self.lib.bpm_surrogate_save(self.ctx.h, self.sid, path.encode()))

    def load(self, path: str):
        L.check(self.lib.bpm_surrogate_load(self.ctx.h, self.sid, path.encode()))

    def destroy(self):
        if self.sid is not None:
            self.lib.bpm_surrogate_destroy(self.ctx.h, self.sid)
            self.sid = None


class Batch:
    def __init__(self, ctx: Context, islands, params, precision, map_id):
        self.ctx = ctx
        self.lib = ctx.lib
        self.isl = island_array(islands)
        self.B = len(self.isl)
        self.n = max(ctx.mesh_info(int(mid))["n_nodes"] for mid in np.unique(self.isl["mesh_id"]))
        self.q = run_params(params, precision, map_id)
        h = c_void_p()
        L.check(self.lib.bpm_batch_create(ctx.h, L.ptr(self.isl), self.B, byref(self.q), byref(h)))
        self.h = h

    def destroy(self):
        if self.h:
            self.lib.bpm_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()

    def set_state(self, m=None, t0_ps: float = 0.0):
        """m: host [B][3][ld] float32 (or a CUDA tensor of that shape), None for +z."""
        on_dev = int(getattr(m, "is_cuda", False))
        if on_dev:
            device_tensor(m, self.ctx.device, "float32", (self.B, 3, None), "m")
        elif m is not None:
            m = np.ascontiguousarray(m, np.float32)
            if m.ndim != 3 or m.shape[:2] != (self.B, 3):
                raise ValueError(f"m: shape {m.shape}, expected ({self.B}, 3, ld)")
        ld = self.n if m is None else int(m.shape[-1])
        with self.ctx.device_order() if on_dev else contextlib.nullcontext():
            L.check(self.lib.bpm_batch_set_state(self.h, L.ptr(m), ld, float(t0_ps), on_dev))

    def advance(self, n_intervals: int):
        L.check(self.lib.bpm_batch_advance(self.h, int(n_intervals)))

    def read(self) -> dict:
        m = np.zeros((self.B, 3, self.n), np.float32)
        sw = np.zeros(self.B, np.uint8)
        tsw = np.zeros(self.B, np.float32)
        st = np.zeros(self.B, np.int32)
        mz = np.zeros(self.B, np.float32)
        L.check(self.lib.bpm_batch_read(self.h, L.ptr(m), self.n, L.ptr(sw), L.ptr(tsw), L.ptr(st), L.ptr(mz), 0))
        return dict(m=m, switched=sw.astype(bool), t_sw=tsw, status=st, mz=mz)

    def read_device(self, m, switched, t_sw, status, mz):
        """Stream-ordered read into device tensors (any may be None): m float32 [B][3][ld],
        switched uint8 [B], t_sw float32 [B], status int32 [B], mz float32 [B]."""
        dev, B = self.ctx.device, self.B
        for t, dt, shape, name in ((m, "float32", (B, 3, None), "m"), (switched, "uint8", (B,), "switched"),
                                   (t_sw, "float32", (B,), "t_sw"), (status, "int32", (B,), "status"),
                                   (mz, "float32", (B,), "mz")):
            if t is not None:
                device_tensor(t, dev, dt, shape, name)
        ld = self.n if m is None else int(m.shape[-1])
        with self.ctx.device_order():
            L.check(self.lib.bpm_batch_read(self.h, L.ptr(m), ld, L.ptr(switched), L.ptr(t_sw), L.ptr(status),
                                            L.ptr(mz), 1))

    def field(self, t_ps: float, term_mask: int) -> np.ndarray:
        out = np.zeros((self.B, 3, self.n), np.float32)
        L.check(self.lib.bpm_batch_field(self.h, float(t_ps), int(term_mask), L.ptr(out), self.n, 0))
        return out

    def energy(self):
        """Energy (J, FP64 accumulation) and largest torque |m x B| (T) of every island
        at the batch's current time (bpm_batch_energy)."""
        E = np.zeros(self.B, np.float64)
        T = np.zeros(self.B, np.float32)
        L.check(self.lib.bpm_batch_energy(self.h, L.ptr(E), L.ptr(T)))
        return E, T

    def kernel_times(self, reps: int = 10) -> dict:
        g, s1, s2 = c_double(), c_double(), c_double()
        L.check(self.lib.bpm_batch_kernel_times(self.h, int(reps), byref(g), byref(s1), byref(s2)))
        return dict(gemm_ms=g.value, stage1_ms=s1.value, stage2_ms=s2.value)

    def graph_kernels(self) -> int:
        """Kernel launches per interval in the batch's CUDA graph."""
        n = c_int32()
        L.check(self.lib.bpm_batch_graph_kernels(self.h, byref(n)))
        return n.value

    def autotune(self, reps: int = 4) -> dict:
        t = L.bpm_tuning()
        L.check(self.lib.bpm_batch_autotune(self.h, int(reps), byref(t)))
        return dict(gemm_tile_n=t.gemm_tile_n, stage_threads=t.stage_threads, gemm_raster=t.gemm_raster,
                    stage_islands=t.stage_islands, gemm_k_block=t.gemm_k_block, gemm_pair=t.gemm_pair,
                    streams=t.streams, gemm_ms=t.gemm_ms, stage_ms=t.stage_ms)

    def set_tuning(self, gemm_tile_n: int, stage_threads: int, gemm_raster: int = L.RASTER_AUTO,
                   stage_islands: int = 1, gemm_k_block: int = 32, gemm_pair: int = 0, streams: int = 2, **_):
        t = L.bpm_tuning(int(gemm_tile_n), int(stage_threads), int(gemm_raster), int(stage_islands),
                         int(gemm_k_block), int(gemm_pair), int(streams), 0.0, 0.0)
        L.check(self.lib.bpm_batch_set_tuning(self.h, byref(t)))

    def tuning_key(self, device_name: str = "") -> str:
        info = [self.ctx.mesh_info(int(mid))["n_pad"] for mid in np.unique(self.isl["mesh_id"])]
        return f"{device_name}|npad={','.join(map(str, info))}|B={self.B}|prec={self.q.precision}"

    def autotune_cached(self, cache_path: str, device_name: str = "", reps: int = 4) -> dict:
        """Apply the tuning cached under this batch's key in a JSON file, or
        autotune, store the choice and apply it."""
        import json
        import os
        key = self.tuning_key(device_name)
        def load():
            try:
                with open(cache_path) as f:
                    return json.load(f)
            except (OSError, ValueError):               # absent, or cut short by another writer
                return {}
        cache = load()
        if key in cache:
            self.set_tuning(**cache[key])
            return dict(cache[key], cached=True)
        t = self.autotune(reps)
        # several processes (one per GPU) may share the file: merge with what is there now and
        # replace it atomically, so that no reader sees a partial write
        cache = load()
        cache[key] = t
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        tmp = f"{cache_path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
        return dict(t, cached=False)

    def time(self) -> float:
        t = c_double()
        L.check(self.lib.bpm_batch_time(self.h, byref(t)))
        return t.value


def substeps_for_bound(field_bound_T: float, dt_ps: float, alpha: float) -> int:
    """The library's step rule (bpm_substeps_for_bound): the smallest k with
    gamma/(1+alpha^2) B dt / k <= 1/2.  Host arithmetic; needs no GPU."""
    k = c_int32()
    L.check(L.load().bpm_substeps_for_bound(float(field_bound_T), float(dt_ps), float(alpha), byref(k)))
    return k.value
