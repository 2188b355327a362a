"""PyTorch-facing wrappers over the C ABI (device memory and streams only).

Tensors passed in must be CUDA float64 and contiguous on the mesh's device; the
direction set (omega [D][2], weights [D]) is given as host arrays.  Outputs are
allocated with torch and filled by the library's kernels.
"""
import ctypes

import numpy as np
import torch

from . import _lib

_NULL = None


def _ptr(t, dtype=torch.float64):
    if t is None:
        return _NULL
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA {str(dtype).replace('torch.', '')} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, shape_last=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _opts(precision="fp64", tol=0.0, max_passes=0, tile=0, groups="direct", kernel="cta", apply="fused",
          pivot="guard", reuse=False):
    o = _lib.VefOpts()
    o.precision = {"fp64": _lib.VEF_FP64, "mixed": _lib.VEF_MIXED}[precision]
    o.tol = float(tol)
    o.max_passes = int(max_passes)
    o.tile_override = int(tile)
    o.flags = {"direct": 0, "iterative": _lib.VEF_GROUPS_ITERATIVE}[groups]
    o.flags |= {"cta": 0, "cluster": _lib.VEF_SWEEP_CLUSTER}[kernel]
    o.flags |= {"fused": 0, "separate": _lib.VEF_APPLY_SEPARATE}[apply]
    o.flags |= {"guard": 0, "always": _lib.VEF_PIVOT_ALWAYS}[pivot]
    o.flags |= _lib.VEF_REUSE_FACTORS if reuse else 0
    return o


def fma_peak(precision="fp64"):
    """Measured FMA throughput (flop/s) of the current device for FP64 or FP32."""
    lib = _lib.load()
    v = ctypes.c_double()
    code = _lib.VEF_FP64 if precision == "fp64" else _lib.VEF_MIXED
    _lib.check(lib.vef_measure_fma_peak(code, ctypes.byref(v)), "vef_measure_fma_peak")
    return v.value


class Mesh:
    """nx x ny mesh of [0,1]^2, Q_m map (sine distortion alpha), DG order p."""

    def __init__(self, nx, ny, mesh_order, p, alpha=0.0, ctrl=None):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        keep = None
        cptr = None
        if ctrl is not None:
            keep, cptr = _host(ctrl)
        _lib.check(self.lib.vef_mesh_create(int(nx), int(ny), int(mesh_order), int(p), float(alpha),
                                            cptr, ctypes.byref(h)), "vef_mesh_create")
        del keep
        self.handle = h
        d = _lib.VefMeshDesc()
        _lib.check(self.lib.vef_mesh_query(h, ctypes.byref(d)), "vef_mesh_query")
        self.nx, self.ny, self.m, self.p = d.nx, d.ny, d.mesh_order, d.p
        self.n, self.nq, self.E, self.nbf = d.n, d.nq, int(d.E), int(d.nbf)
        self.device = torch.cuda.current_device()

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.vef_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable=True):
        """Turn per-kernel CUDA-event timing on/off (resets the counters)."""
        _lib.check(self.lib.vef_profile(self.handle, int(bool(enable))), "vef_profile")

    def profile_read(self):
        """{kernel class: (launches, summed ms)} since the last vef_profile call."""
        arr = (_lib.VefKernelStat * len(_lib.KERNEL_CLASSES))()
        _lib.check(self.lib.vef_profile_read(self.handle, arr), "vef_profile_read")
        return {k: (arr[i].launches, arr[i].ms) for i, k in enumerate(_lib.KERNEL_CLASSES)}

    def sync(self, stream=None):
        _lib.check(self.lib.vef_mesh_sync(self.handle, _stream(stream)), "vef_mesh_sync")

    def _empty(self, *shape):
        return torch.empty(*shape, dtype=torch.float64, device=f"cuda:{self.device}")

    # ---------------------------------------------------------------- transport
    def sweep(self, sigma_t, sigma_s, omega, weights, phi_in=None, source=None, inflow=None,
              precision="fp64", tol=0.0, max_passes=0, tile=0, groups="direct", psi=None, info=False,
              stream=None, kernel="cta", apply="fused", pivot="guard", reuse=False):
        """psi [D][E][n] = L^{-1} b for every direction (see vef_sweep in include/vef.h).

        groups: "direct" (coupled element groups through their trace system) or
        "iterative" (inner block Gauss-Seidel for every group).
        kernel: "cta" (one CTA per direction, the default) or "cluster" (a thread-block
        cluster per direction; a nonzero tile also selects it).
        apply: "fused" (y = A^{-1} b computed inside the sweep launch on the SMs the
        directions leave free, when enough are free and the stream is not being captured)
        or "separate" (its own launch before the sweep); both give the same psi.
        pivot: "guard" (element systems eliminated without pivoting, those meeting a small
        pivot redone with partial pivoting) or "always" (every system with partial
        pivoting; slow, for tests).
        reuse: keep the local factorisation of the previous call with this direction set and
        precision (the caller guarantees sigma_t is unchanged)."""
        om, omp = _host(omega)
        w, wp = _host(weights)
        D = len(w)
        aniso = int(source is not None and source.dim() == 3)
        if psi is None:
            psi = self._empty(D, self.E, self.n)
        inf = _lib.VefInfo() if info else None
        o = _opts(precision, tol, max_passes, tile, groups, kernel, apply, pivot, reuse)
        st = self.lib.vef_sweep(self.handle, _ptr(sigma_t), _ptr(sigma_s), _ptr(phi_in), _ptr(source),
                                aniso, _ptr(inflow), omp, wp, D, ctypes.byref(o), _ptr(psi),
                                ctypes.byref(inf) if info else None, _stream(stream))
        _lib.check(st, "vef_sweep")
        return (psi, inf.as_dict()) if info else psi

    def moments(self, psi, omega, weights, inflow=None, outputs=("phi", "J", "P", "E", "Eb", "Jin"),
                stream=None):
        """dict of phi [E][n], J [2][E][n], P [3][E][n], E [3][E][nq^2], Eb, Jin [N_bf][nq]."""
        om, omp = _host(omega)
        w, wp = _host(weights)
        D = len(w)
        out = {}
        shapes = {"phi": (self.E, self.n), "J": (2, self.E, self.n), "P": (3, self.E, self.n),
                  "E": (3, self.E, self.nq * self.nq), "Eb": (self.nbf, self.nq),
                  "Jin": (self.nbf, self.nq)}
        for k in outputs:
            out[k] = self._empty(*shapes[k])
        st = self.lib.vef_moments(self.handle, _ptr(psi), omp, wp, D, _ptr(inflow),
                                  _ptr(out.get("phi")), _ptr(out.get("J")), _ptr(out.get("P")),
                                  _ptr(out.get("E")), _ptr(out.get("Eb")), _ptr(out.get("Jin")),
                                  _stream(stream))
        _lib.check(st, "vef_moments")
        return out

    def source_iterate(self, sigma_t, sigma_s, omega, weights, K, source=None, inflow=None, phi0=None,
                       precision="fp64", tol=0.0, max_passes=0, psi=None, info=False, stream=None,
                       kernel="cta"):
        """K source iterations: returns (phi^K, psi of the last sweep, dphi_inf [K])."""
        om, omp = _host(omega)
        w, wp = _host(weights)
        D = len(w)
        aniso = int(source is not None and source.dim() == 3)
        if psi is None:
            psi = self._empty(D, self.E, self.n)
        phi = self._empty(self.E, self.n)
        dphi = self._empty(K)
        inf = _lib.VefInfo() if info else None
        o = _opts(precision, tol, max_passes, kernel=kernel)
        st = self.lib.vef_source_iterate(self.handle, _ptr(sigma_t), _ptr(sigma_s), _ptr(phi0),
                                         _ptr(source), aniso, _ptr(inflow), omp, wp, D, int(K),
                                         ctypes.byref(o), _ptr(phi), _ptr(psi), _ptr(dphi),
                                         ctypes.byref(inf) if info else None, _stream(stream))
        _lib.check(st, "vef_source_iterate")
        return (phi, psi, dphi, inf.as_dict()) if info else (phi, psi, dphi)

    def hrt_solve(self, sigma_t, sigma_s, phi_tr, P_tr, Eb, Jin, Q0, Q1=None, tol=1e-13, max_iter=2000,
                  check=True, stream=None):
        """Hybridized RT VEF solve (see vef_hrt_solve in include/vef.h): returns
        (phi [E][n], J [E][2 (p+2)(p+1)], lambda [faces][p+1], info dict).  check=False
        returns the last iterate with info["converged"] = False instead of raising when the
        multiplier solve stops at max_iter."""
        nJ = 2 * (self.p + 2) * (self.p + 1)
        nfaces = (self.nx - 1) * self.ny + self.nx * (self.ny - 1)
        phi = self._empty(self.E, self.n)
        J = self._empty(self.E, nJ)
        lam = self._empty(max(nfaces, 1), self.p + 1)
        inf = _lib.VefHrtInfo()
        st = self.lib.vef_hrt_solve(self.handle, _ptr(sigma_t), _ptr(sigma_s), _ptr(phi_tr), _ptr(P_tr),
                                    _ptr(Eb), _ptr(Jin), _ptr(Q0), _ptr(Q1), float(tol), int(max_iter),
                                    _ptr(phi), _ptr(J), _ptr(lam), ctypes.byref(inf), _stream(stream))
        if check or st != _lib.VEF_ERR_NOT_CONVERGED:
            _lib.check(st, "vef_hrt_solve")
        d = inf.as_dict()
        d["converged"] = st == _lib.VEF_OK
        return phi, J, lam[:nfaces], d

    def vef_iterate(self, sigma_t, sigma_s, omega, weights, source=None, inflow=None, phi0=None, max_outer=50,
                    tol=1e-6, hrt_tol=1e-12, hrt_max_iter=5000, precision="fp64", psi=None, check=True,
                    stream=None):
        """VEF fixed-point iteration (see vef_vef_iterate in include/vef.h): returns
        (phi [E][n], J [E][2 (p+2)(p+1)], psi [D][E][n], dphi [iterations], info dict)."""
        om, omp = _host(omega)
        w, wp = _host(weights)
        D = len(w)
        nJ = 2 * (self.p + 2) * (self.p + 1)
        phi = self._empty(self.E, self.n)
        J = self._empty(self.E, nJ)
        if psi is None:
            psi = self._empty(D, self.E, self.n)
        dphi = self._empty(max_outer)
        inf = _lib.VefVefInfo()
        o = _opts(precision)
        st = self.lib.vef_vef_iterate(self.handle, _ptr(sigma_t), _ptr(sigma_s), _ptr(source), _ptr(inflow), omp,
                                      wp, D, _ptr(phi0), int(max_outer), float(tol), float(hrt_tol),
                                      int(hrt_max_iter), ctypes.byref(o), _ptr(phi), _ptr(J), _ptr(psi),
                                      _ptr(dphi), ctypes.byref(inf), _stream(stream))
        if check or st != _lib.VEF_ERR_NOT_CONVERGED:
            _lib.check(st, "vef_vef_iterate")
        d = inf.as_dict()
        return phi, J, psi, dphi[:d["iterations"]], d

    def region_weights(self, lo=(0.6, 0.6), hi=(0.8, 0.8), stream=None):
        """g [E][n] with sum g * phi = int over the box [lo, hi] of phi dx."""
        g = self._empty(self.E, self.n)
        _lib.check(self.lib.vef_region_weights(self.handle, float(lo[0]), float(lo[1]), float(hi[0]),
                                               float(hi[1]), _ptr(g), _stream(stream)), "vef_region_weights")
        return g

    def adjoint(self, sigma_t, sigma_s, omega, weights, psi, g, phi_in=None, want_lambda=False,
                info=False, stream=None, kernel="cta"):
        """Gradients of R = sum g * phi: returns (dR/dsigma_t [E], dR/dsigma_s [E] or None, lambda).

        psi: the forward sweep's psi [D][E][n] as checkpoint, float64, or float32 (an FP32
        copy, half the memory; the gradients then carry its rounding).
        kernel: "cta" (one CTA per direction, the default) or "cluster"."""
        om, omp = _host(omega)
        w, wp = _host(weights)
        D = len(w)
        lam = self._empty(D, self.E, self.n) if want_lambda else None
        dst = self._empty(self.E)
        dss = self._empty(self.E) if phi_in is not None else None
        inf = _lib.VefInfo() if info else None
        o = _opts(kernel=kernel)
        if psi.dtype == torch.float32:
            o.flags |= _lib.VEF_CKPT_FP32
        elif psi.dtype != torch.float64:
            raise TypeError("psi checkpoint must be float64 or float32")
        st = self.lib.vef_adjoint_sweep(self.handle, _ptr(sigma_t), _ptr(sigma_s), _ptr(phi_in), omp,
                                        wp, D, _ptr(psi, psi.dtype), _ptr(g), _ptr(lam), _ptr(dst), _ptr(dss),
                                        ctypes.byref(o), ctypes.byref(inf) if info else None, _stream(stream))
        _lib.check(st, "vef_adjoint_sweep")
        res = (dst, dss, lam)
        return res + (inf.as_dict(),) if info else res


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for k, t in enumerate(items):
        arr[k] = None if t is None else _ptr(t).value
    return arr


class Batch:
    """Independent problems swept together (one cluster launch per DG order)."""

    def __init__(self, meshes, omegas, weights):
        self.lib = _lib.load()
        self.meshes = list(meshes)
        self._om = [np.ascontiguousarray(np.asarray(o, np.float64)) for o in omegas]
        self._w = [np.ascontiguousarray(np.asarray(w, np.float64)) for w in weights]
        n = len(self.meshes)
        mh = (ctypes.c_void_p * n)(*[m.handle.value for m in self.meshes])
        op = (ctypes.c_void_p * n)(*[o.ctypes.data for o in self._om])
        wp = (ctypes.c_void_p * n)(*[w.ctypes.data for w in self._w])
        D = (ctypes.c_int * n)(*[len(w) for w in self._w])
        h = ctypes.c_void_p()
        _lib.check(self.lib.vef_batch_create(mh, n, op, wp, D, ctypes.byref(h)), "vef_batch_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.vef_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, sigma_t, sigma_s, phi_in=None, source=None, inflow=None, psi=None, tile=0,
              info=False, stream=None, reuse=False):
        """Lists of per-problem tensors; returns the list of psi [D_k][E_k][n_k].
        tile: 0 = the tuned (or default single-CTA) form, else a cluster shape 100 x CTAs +
        warps; reuse: keep the previous call's factorisations (sigma_t unchanged)."""
        n = len(self.meshes)
        if psi is None:
            psi = [m._empty(len(w), m.E, m.n) for m, w in zip(self.meshes, self._w)]
        none = lambda lst: None if lst is None else _ptr_array(lst)
        o = _opts("fp64", 0.0, 0, tile, reuse=reuse)
        inf = _lib.VefInfo() if info else None
        st = self.lib.vef_batch_sweep(self.handle, _ptr_array(sigma_t), _ptr_array(sigma_s), none(phi_in),
                                      none(source), none(inflow), _ptr_array(psi), ctypes.byref(o),
                                      ctypes.byref(inf) if info else None, _stream(stream))
        _lib.check(st, "vef_batch_sweep")
        return (psi, inf.as_dict()) if info else psi

    def tune(self, stream=None):
        """Autotune the sweep form per DG order; returns {p: tile} (1 = one CTA per
        (problem, direction), else 100 x CTAs per cluster + warps per CTA)."""
        tiles = (ctypes.c_int * 4)()
        _lib.check(self.lib.vef_batch_tune(self.handle, _stream(stream), tiles), "vef_batch_tune")
        return {p + 1: tiles[p] for p in range(4) if tiles[p]}
