"""GB300-native range-separated (RS) canonical/Tucker tensor method for the N-particle
Newton potential (Benner, Khoromskaia, Khoromskij, arXiv:1606.09218).

The computation runs in ``librs_gb300.so`` (hand-written CUDA for sm_103a behind the C ABI of
``include/rs.h``).  This module only marshals arguments: PyTorch supplies device memory
and streams.
"""
from __future__ import annotations

import ctypes as C

from . import _lib
from ._lib import (RS_ENERGY, RS_FORCES, RS_FORCES_PAIR, RS_FP32, RS_FP32_SPLIT, RS_FP64,  # noqa: F401
                   RS_INPUT_HOST, RS_POTENTIAL, RS_VALIDATE_SEPARATION, RSError)

PRECISIONS = {"fp64": RS_FP64, "fp32_split": RS_FP32_SPLIT, "fp32": RS_FP32}


def config_from_workload(cfg: dict, n: int | None = None, max_particles: int | None = None,
                         max_rank: int = 0) -> _lib.RSConfigC:
    """Build the C config from a workload parameter dictionary."""
    c = _lib.RSConfigC()
    nn = int(n if n is not None else cfg["n"])
    if "quad_by_n" in cfg:
        q = cfg["quad_by_n"][str(nn)]
        hq, u0 = q["h_q"], q["u0"]
    else:
        hq, u0 = cfg["h_q"], cfg["u0"]
    c.b = float(cfg["b"])
    c.n = nn
    c.R = int(cfg["R"])
    c.R_s = int(cfg["R_s"])
    c.h_q = float(hq)
    c.u0 = float(u0)
    c.eps = float(cfg["eps"])
    c.rank_cap = int(cfg.get("rank_cap", 0))
    c.max_rank = int(max_rank or cfg.get("max_rank", 0))
    c.delta_rel = float(cfg["delta_rel"])
    c.precision = PRECISIONS[cfg.get("precision", "fp32_split")]
    c.snap = 1 if cfg.get("snap", True) else 0
    if max_particles is None:
        max_particles = int(cfg.get("particles", {}).get("N", 0)) or 1
        if cfg.get("particles", {}).get("kind") == "nacl_lattice":
            max_particles = int(cfg["particles"]["side"]) ** 3
    c.max_particles = int(max_particles)
    return c


class _DevArray:
    """Exposes a library-owned device buffer through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str, strides=None):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3, "strides": strides}


class RSContext:
    """One device context of the library (workspace sized for ``cfg``)."""

    def __init__(self, cfg: _lib.RSConfigC, stream=None):
        import torch
        self._torch = torch
        self.lib = _lib.load()
        self.cfg = cfg
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.rs_create(C.byref(cfg), C.c_void_p(stream.cuda_stream), C.byref(h))
        _lib.check(st, None)
        self.h = h
        self.n = cfg.n
        self.fp64 = cfg.precision == RS_FP64
        self.dtype = torch.float64 if self.fp64 else torch.float32

    def close(self):
        if getattr(self, "h", None):
            self.lib.rs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_potential(self):
        n = self.n
        return self._torch.empty((n, n, n), dtype=self.dtype, device="cuda")

    def solve(self, xyz, Z, potential=None, energy: bool = True, want_potential: bool = True,
              min_sep: float = 0.0, forces: bool = False, forces_pair: bool = False) -> int:
        """Enqueue one solve.  ``xyz`` (N,3) and ``Z`` (N,) float64: CUDA tensors, or host
        (CPU tensors / numpy) which the library copies in.  ``forces``: the discrete gradient of
        the RS-Tucker tensor; with ``forces_pair`` the long part from the untruncated pair
        kernel instead.  Returns the launch status."""
        torch = self._torch
        flags = 0
        if isinstance(xyz, torch.Tensor) and xyz.is_cuda:
            assert xyz.dtype == torch.float64 and Z.dtype == torch.float64
            xyz = xyz.contiguous()
            Z = Z.contiguous()
            pxyz, pZ = xyz.data_ptr(), Z.data_ptr()
            N = int(Z.numel())
            self._keep = (xyz, Z)
        else:
            import numpy as np
            xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64))
            Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64))
            pxyz, pZ = xyz.ctypes.data, Z.ctypes.data
            N = int(Z.size)
            flags |= RS_INPUT_HOST
            self._keep = (xyz, Z)
        out = 0
        if want_potential:
            if potential is None:
                potential = self.new_potential()
            assert potential.dtype == self.dtype and potential.is_cuda and potential.numel() == self.n ** 3
            out = potential.data_ptr()
            flags |= RS_POTENTIAL
        if energy:
            flags |= RS_ENERGY
        if forces:
            flags |= RS_FORCES
            if forces_pair:
                flags |= RS_FORCES_PAIR
        self.last_N = N
        if min_sep > 0:
            flags |= RS_VALIDATE_SEPARATION
        st = self.lib.rs_solve(self.h, N, C.c_void_p(pxyz), C.c_void_p(pZ), flags, float(min_sep),
                               C.c_void_p(out))
        _lib.check(st, self.h)
        self.potential = potential
        return st

    def energy(self) -> float:
        E = C.c_double()
        _lib.check(self.lib.rs_energy(self.h, C.byref(E)), self.h)
        return float(E.value)

    def forces(self):
        """Forces of the last solve (it must have asked for ``forces=True``) as an (N, 3)
        float64 CUDA tensor (Sec. 4.3): the discrete gradient of the RS-Tucker tensor (or the
        untruncated pair kernel with ``forces_pair``), the windows term by term."""
        torch = self._torch
        F = torch.empty((self.last_N, 3), dtype=torch.float64, device="cuda")
        _lib.check(self.lib.rs_forces(self.h, C.c_void_p(F.data_ptr()), 0), self.h)
        return F

    def pair_energy_forces(self, xyz, Z, forces: bool = True):
        """Energy (and forces) of centres anywhere in the box with the RS kernel in pair form
        (rs_pair_energy_forces); xyz (N, 3) and Z (N,) float64 CUDA tensors.  Returns
        (E, F) with F an (N, 3) float64 CUDA tensor or None."""
        torch = self._torch
        xyz = xyz.contiguous()
        Z = Z.contiguous()
        assert xyz.is_cuda and Z.is_cuda and xyz.dtype == torch.float64 and Z.dtype == torch.float64
        N = int(Z.numel())
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.empty((N, 3), dtype=torch.float64, device="cuda") if forces else None
        _lib.check(self.lib.rs_pair_energy_forces(self.h, N, C.c_void_p(xyz.data_ptr()), C.c_void_p(Z.data_ptr()),
                                                  C.c_void_p(E.data_ptr()),
                                                  C.c_void_p(F.data_ptr()) if F is not None else None), self.h)
        return float(E.item()), F

    def matvec(self, X, Y=None, long: bool = True, short: bool = True, offdiag: bool = False):
        """Y = A X with the RS interaction matrix of the grid (rs_matvec; Sec. 4.1, case (A)):
        X an (n, n, n) CUDA tensor of the context's dtype; returns Y (a new tensor if None)."""
        torch = self._torch
        X = X.contiguous()
        assert X.is_cuda and X.dtype == self.dtype and X.numel() == self.n ** 3
        if Y is None:
            Y = torch.empty_like(X)
        flags = (_lib.RS_MATVEC_LONG if long else 0) | (_lib.RS_MATVEC_SHORT if short else 0)
        if not (long or short):
            raise ValueError("select the long terms, the short terms or both")
        if offdiag:
            flags |= _lib.RS_MATVEC_OFFDIAG
        _lib.check(self.lib.rs_matvec(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()), flags), self.h)
        return Y

    def energy_matvec(self) -> float:
        """E_N = 1/2 <(A - diag A) z, z> of the last solve's charges through the interaction
        matrix (rs_energy_matvec; Sec. 4.2, Eq. (4.6))."""
        E = C.c_double()
        _lib.check(self.lib.rs_energy_matvec(self.h, C.byref(E)), self.h)
        return float(E.value)

    def plain_direct(self, out=None):
        """Direct sum sum_nu Z_nu / |x - x_nu| of the last solve's particles on the grid
        (plain-method GPU path, no RS format); returns the (n, n, n) float32 CUDA tensor."""
        return self._plain(self.lib.rs_plain_direct, out)

    def plain_canonical(self, out=None):
        """Full-rank canonical sum P_0 of the last solve's particles on the grid (plain-method
        GPU path: all R terms, no split, no truncation); (n, n, n) float32 CUDA tensor."""
        return self._plain(self.lib.rs_plain_canonical, out)

    def _plain(self, fn, out):
        torch = self._torch
        if out is None:
            out = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        assert out.dtype == torch.float32 and out.is_cuda and out.numel() == self.n ** 3
        _lib.check(fn(self.h, C.c_void_p(out.data_ptr())), self.h)
        return out

    def report(self) -> dict:
        s = _lib.RSStatsC()
        st = self.lib.rs_report(self.h, C.byref(s))
        _lib.check(st, self.h)
        return dict(N=s.N, N_nonzero=s.N_nonzero, ranks=list(s.ranks), subspace=list(s.subspace),
                    gamma=s.gamma, tail_rel=list(s.tail_rel), eps_bound=s.eps_bound, P_R0=s.P_R0,
                    P_Rl0=s.P_Rl0, energy=s.energy, status=s.status, kernel_launches=s.kernel_launches)

    def profile(self, enable: bool = True):
        """Turn per-stage CUDA-event timing on or off."""
        _lib.check(self.lib.rs_profile_enable(self.h, 1 if enable else 0), self.h)

    def profile_read(self) -> tuple[dict, int]:
        """Per-stage device milliseconds summed over the solves since the last read."""
        ms = (C.c_double * _lib.RS_NSTAGE)()
        cnt = C.c_int()
        _lib.check(self.lib.rs_profile_read(self.h, ms, C.byref(cnt)), self.h)
        names = [self.lib.rs_stage_name(i).decode() for i in range(_lib.RS_NSTAGE)]
        return {nm: ms[i] for i, nm in enumerate(names)}, cnt.value

    def tucker(self):
        """(ranks, [V1, V2, V3], beta) as torch views of the library's buffers (valid until
        the next solve); V_l is n x r_l, beta is r1 x r2 x r3."""
        torch = self._torch
        ranks = (C.c_int * 3)()
        ldV, ldb = C.c_int(), C.c_int()
        V = (C.c_void_p * 3)()
        beta = C.c_void_p()
        _lib.check(self.lib.rs_get_tucker(self.h, ranks, C.byref(ldV), C.byref(ldb), V, C.byref(beta)),
                   self.h)
        ts = "<f8" if self.fp64 else "<f4"
        es = 8 if self.fp64 else 4
        n = self.n
        Vs = []
        for l in range(3):
            full = torch.as_tensor(_DevArray(V[l], (n, ldV.value), ts), device="cuda")
            Vs.append(full[:, : ranks[l]])
        bfull = torch.as_tensor(_DevArray(beta.value, (ldb.value,) * 3, ts), device="cuda")
        del es
        return list(ranks), Vs, bfull[: ranks[0], : ranks[1], : ranks[2]]

    def windows(self):
        """Short-range part of the last solve (rs_get_windows; Defs. 3.4, 3.6): (gamma, factors
        (R_s, n_s) float64, grid indices (N, 3) int32, charges (N,) float64) as torch views of
        the library's buffers (valid until the next solve)."""
        torch = self._torch
        ns, rs_, N, ld = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        f, j, z = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _lib.check(self.lib.rs_get_windows(self.h, C.byref(ns), C.byref(rs_), C.byref(N), C.byref(f), C.byref(ld),
                                           C.byref(j), C.byref(z)), self.h)
        R_s, n_s, L, NN = rs_.value, ns.value, ld.value, N.value
        fac = torch.as_tensor(_DevArray(f.value, (R_s, n_s), "<f8", strides=(8 * L, 8)), device="cuda")
        if NN > 0:
            jj = torch.as_tensor(_DevArray(j.value, (NN, 3), "<i4"), device="cuda")
            zz = torch.as_tensor(_DevArray(z.value, (NN,), "<f8"), device="cuda")
        else:
            jj = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
            zz = torch.zeros(0, dtype=torch.float64, device="cuda")
        return (n_s - 1) // 2, fac, jj, zz

    def debug_buffer(self, name: str, dtype=None):
        """A torch (uint8 or ``dtype``) view of an internal device buffer (inspection hook)."""
        torch = self._torch
        ptr, nb = C.c_void_p(), C.c_size_t()
        _lib.check(self.lib.rs_debug_buffer(self.h, name.encode(), C.byref(ptr), C.byref(nb)), self.h)
        raw = torch.as_tensor(_DevArray(ptr.value, (nb.value,), "|u1"), device="cuda")
        return raw if dtype is None else raw.view(dtype)

    def canonical(self, eps: float) -> int:
        """RS-canonical form of the last solve (Def. 3.7): Tucker-to-canonical transform of the
        long part at accuracy ``eps`` (slice SVD of the core); returns the canonical rank R*."""
        r = C.c_int()
        _lib.check(self.lib.rs_canonical(self.h, float(eps), C.byref(r)), self.h)
        return int(r.value)

    def canonical_eval_points(self, idx):
        """RS-canonical entries (Lemma 3.8) at grid multi-indices idx (M,3) int32 CUDA tensor."""
        torch = self._torch
        idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(idx.shape[0], dtype=torch.float64, device="cuda")
        _lib.check(self.lib.rs_canonical_eval_points(self.h, int(idx.shape[0]), C.c_void_p(idx.data_ptr()),
                                                     C.c_void_p(out.data_ptr())), self.h)
        return out

    def tucker_als(self, sweeps: int = 1, energy: bool = True, potential=None, want_potential: bool = True) -> int:
        """ALS refinement of the last solve's canonical-to-Tucker transform (Sec. 6, steps
        (III)-(V)): ``sweeps`` sweeps over the modes with eps-truncated ranks.  With
        ``want_potential`` the refined full-grid potential is written to ``potential`` (a new
        tensor if None, kept as ``self.potential``); with ``energy`` the energy is recomputed."""
        flags = RS_ENERGY if energy else 0
        out = 0
        if want_potential:
            if potential is None:
                potential = self.new_potential()
            assert potential.dtype == self.dtype and potential.is_cuda and potential.numel() == self.n ** 3
            out = potential.data_ptr()
            flags |= RS_POTENTIAL
        st = self.lib.rs_tucker_als(self.h, int(sweeps), flags, C.c_void_p(out))
        _lib.check(st, self.h)
        if want_potential:
            self.potential = potential
        return st

    def get_canonical(self):
        """(xi (R*,), [U1, U2, U3] (n, R*)) float64 CUDA views of the RS-canonical form."""
        torch = self._torch
        r, xi, U, ld = C.c_int(), C.c_void_p(), C.c_void_p(), C.c_int()
        _lib.check(self.lib.rs_get_canonical(self.h, C.byref(r), C.byref(xi), C.byref(U), C.byref(ld)), self.h)
        R, n, L = int(r.value), self.n, int(ld.value)
        xi_t = torch.as_tensor(_DevArray(xi.value, (max(R, 1),), "<f8"), device="cuda")[:R]
        Uall = torch.as_tensor(_DevArray(U.value, (3 * n * L,), "<f8"), device="cuda").view(3, n, L)[:, :, :R]
        return xi_t, [Uall[0], Uall[1], Uall[2]]

    def eval_points(self, idx):
        """RS-Tucker entries (Lemma 3.10) at grid multi-indices idx (M,3) int32 CUDA tensor."""
        torch = self._torch
        idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(idx.shape[0], dtype=torch.float64, device="cuda")
        _lib.check(self.lib.rs_eval_points(self.h, int(idx.shape[0]), C.c_void_p(idx.data_ptr()),
                                           C.c_void_p(out.data_ptr())), self.h)
        return out


def version() -> str:
    return _lib.load().rs_version().decode()


class RSServer:
    """Continuous-batching request loop of the library (``rs_server_*``): requests of any
    configuration are queued by ``submit`` and run concurrently as slots and HBM budget allow."""

    def __init__(self, hbm_budget: int = 32 << 30, max_slots: int = 8):
        self.lib = _lib.load()
        h = C.c_void_p()
        _lib.check(self.lib.rs_server_create(C.c_size_t(int(hbm_budget)), int(max_slots), C.byref(h)), None)
        self.h = h

    def submit(self, cfg: _lib.RSConfigC, xyz, Z, energy: bool = True, potential=None) -> int:
        """Queue one solve (host inputs, copied by the library); returns its ticket."""
        import numpy as np
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64))
        Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64))
        req = _lib.RSRequestC()
        req.cfg = cfg
        req.N = int(Z.size)
        req.xyz = xyz.ctypes.data
        req.Z = Z.ctypes.data
        req.flags = (RS_ENERGY if energy else 0) | (RS_POTENTIAL if potential is not None else 0)
        req.potential_out = potential.data_ptr() if potential is not None else None
        t = C.c_ulonglong()
        _lib.check(self.lib.rs_submit(self.h, C.byref(req), C.byref(t)), None)
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = 120000) -> dict:
        r = _lib.RSResultC()
        _lib.check(self.lib.rs_wait(self.h, C.c_ulonglong(ticket), int(timeout_ms), C.byref(r)), None)
        return dict(status=r.status, energy=r.energy, latency_ms=r.latency_ms, queue_ms=r.queue_ms,
                    ranks=list(r.ranks), slot=r.slot, message=r.message.decode(errors="replace"))

    def info(self) -> dict:
        sl, q = C.c_int(), C.c_int()
        b = C.c_size_t()
        _lib.check(self.lib.rs_server_info(self.h, C.byref(sl), C.byref(b), C.byref(q)), None)
        return dict(slots=sl.value, bytes_in_use=b.value, queued=q.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.rs_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _energy_function():
    import torch

    class RSEnergy(torch.autograd.Function):
        """E(xyz) of the RS-Tucker tensor with the forces as the gradient: dE/dxyz = -F, the
        discrete gradient (Sec. 4.3, Eq. (4.9)) of the same tensor whose energy forward returns."""

        @staticmethod
        def forward(fctx, xyz, Z, rs):
            rs.solve(xyz.detach(), Z.detach(), energy=True, want_potential=False, forces=True)
            E = rs.energy()
            F = rs.forces()
            fctx.save_for_backward(F)
            return torch.tensor(E, dtype=torch.float64, device=xyz.device)

        @staticmethod
        def backward(fctx, gE):
            (F,) = fctx.saved_tensors
            return -gE * F, None, None

    return RSEnergy


def rs_energy(xyz, Z, ctx: RSContext):
    """Differentiable interaction energy: ``rs_energy(xyz, Z, ctx).backward()`` puts -F into
    ``xyz.grad`` (Sec. 4.3 forces through the C ABI)."""
    return _energy_function().apply(xyz, Z, ctx)
