"""Thin PyTorch-facing binding of the C ABI: checks tensors, passes raw device pointers.

Every computation runs in libptim.so; this module only marshals arguments.  The
names follow the C entry points (pt_apply_exchange -> Context.apply_exchange ...).
Orbital blocks are torch tensors of shape (N, nz, ny, nx), complex128 for
precision "fp64" and complex64 for the FP32 forms, on the context's device.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L

_CDTYPE = {"fp64": torch.complex128, "fp32": torch.complex64, "tf32": torch.complex64, "bf16": torch.complex64}


class PtimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _grid(cell) -> L.pt_grid:
    n, Ls = cell.n, cell.L
    g = L.pt_grid()
    g.nx, g.ny, g.nz = int(n[0]), int(n[1]), int(n[2])
    g.L[0], g.L[1], g.L[2] = float(Ls[0]), float(Ls[1]), float(Ls[2])
    return g


def _kernel(kernel) -> L.pt_kernel:
    k = L.pt_kernel()
    kernel = kernel or {"type": 1, "mu": 0.106}
    k.type = int(kernel.get("type", 1))
    k.mu = float(kernel.get("mu", 0.106))
    k.g0 = float(kernel.get("g0", math.nan))
    return k


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _points(cell) -> int:
    return int(cell.n[0]) * int(cell.n[1]) * int(cell.n[2])


def _sized(t: torch.Tensor, count: int, what: str, where: str = "", how: str = ""):
    """Buffers the C ABI reads or writes by pointer must hold exactly what the call addresses
    (the library cannot see tensor sizes; a short buffer would be read or written past its end)."""
    if t.numel() != count:
        raise PtimError(L.PT_INVALID_ARG,
                        f"{where}{what} holds {t.numel()} elements where the call addresses {count}{how}")


def _block(t: torch.Tensor, cell, what: str, where: str = ""):
    """An (N, nz, ny, nx) orbital block on the cell's grid."""
    n = _points(cell)
    _sized(t, t.shape[0] * n, what, where, f" ({t.shape[0]} orbitals x {n} grid points of the cell)")


def _result(out: torch.Tensor, count: int, dtype, device, what: str = "out", where: str = ""):
    """A caller-supplied output: contiguous, of the call's type and device, `count` elements."""
    if out.device != device or out.dtype != dtype or not out.is_contiguous():
        raise ValueError(f"{where}{what} must be a contiguous {dtype} tensor on {device}")
    _sized(out, count, what, where)


def _vec3(A):
    """A host double[3] for an optional 3-vector argument (None -> NULL)."""
    if A is None:
        return None
    a = [float(v) for v in A]
    if len(a) != 3:
        raise ValueError("A must have 3 components")
    return (C.c_double * 3)(*a)


class Ace:
    """Library-owned ACE operator (xi vectors live in device memory until close())."""

    def __init__(self, ctx, handle, N, cell, precision):
        self.ctx, self.handle, self.N, self.cell, self.precision = ctx, handle, N, cell, precision

    def xi(self, stream=None):
        out = torch.empty((self.N, self.cell.n[2], self.cell.n[1], self.cell.n[0]), dtype=_CDTYPE[self.precision],
                          device=self.ctx.device)
        st = L.load().pt_ace_get_xi(self.handle, _ptr(out), _stream(stream))
        if st != L.PT_OK:
            raise PtimError(st, "pt_ace_get_xi failed")
        return out

    def close(self):
        if self.handle:
            L.load().pt_ace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A pt_ctx on one CUDA device (owns workspace and cached tables)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the PT-IM library needs a CUDA GPU; no CPU fallback exists")
        self.lib = L.load()
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        st = self.lib.pt_create(C.byref(h), device, hbm_budget)
        if st != L.PT_OK:
            raise PtimError(st, "pt_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.pt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != L.PT_OK:
            raise PtimError(st, f"{what}: {self.lib.pt_last_error(self.h).decode()}")

    def _orb(self, t, precision, what):
        if t.device != self.device or not t.is_contiguous() or t.dtype != _CDTYPE[precision] or t.dim() != 4:
            raise ValueError(f"{what} must be a contiguous {_CDTYPE[precision]} (N, nz, ny, nx) tensor on {self.device}")
        return t

    def alu_peaks(self, stream=None) -> dict:
        """FP32 and FP64 FMA throughput of the device, TFLOP/s (synchronises the stream)."""
        f32, f64 = C.c_double(0.0), C.c_double(0.0)
        self._check(self.lib.pt_alu_peaks(self.h, C.byref(f32), C.byref(f64), _stream(stream)), "pt_alu_peaks")
        return {"fp32_tflops": f32.value, "fp64_tflops": f64.value}

    def selftest_wait(self, arrive: bool, timeout_s: float = 0.05, stream=None) -> str:
        """Bounded device-wait self-test: the status name, "PT_TIMEOUT" when nothing arrives
        (the expected outcome with arrive=False), "PT_OK" when the barrier completes."""
        st = self.lib.pt_selftest_wait(self.h, int(bool(arrive)), float(timeout_s), _stream(stream))
        if st not in (L.PT_OK, L.PT_TIMEOUT):
            self._check(st, "pt_selftest_wait")
        return L.STATUS_NAMES[st]

    def workspace_bytes(self) -> int:
        return int(self.lib.pt_workspace_bytes(self.h))

    def set_option(self, key: str, value: float):
        self._check(self.lib.pt_set_option(self.h, key.encode(), float(value)), "pt_set_option")

    def trim(self):
        self._check(self.lib.pt_trim(self.h), "pt_trim")

    # ---- exchange --------------------------------------------------------------------------
    def apply_exchange(self, src, occ, tgt=None, out=None, *, cell, kernel=None, precision="fp64", stream=None):
        """out_j = V_x tgt_j = -sum_i occ_i src_i IFFT[K FFT[conj(src_i) tgt_j]] (tgt None: tgt = src)."""
        self._orb(src, precision, "src")
        if tgt is not None:
            self._orb(tgt, precision, "tgt")
        occ = occ.to(device=self.device, dtype=torch.float64).contiguous()
        ref = src if tgt is None else tgt
        _block(src, cell, "src")
        if tgt is not None:
            _block(tgt, cell, "tgt")
        if occ.numel() < src.shape[0]:
            raise PtimError(L.PT_INVALID_ARG, f"occ holds {occ.numel()} occupations for {src.shape[0]} orbitals")
        if out is None:
            out = torch.empty_like(ref)
        _result(out, ref.numel(), ref.dtype, self.device)
        g, k = _grid(cell), _kernel(kernel)
        st = self.lib.pt_apply_exchange(self.h, _ptr(src), _ptr(occ), src.shape[0],
                                        None if tgt is None else _ptr(tgt), ref.shape[0], _ptr(out),
                                        C.byref(g), C.byref(k), L.PRECISIONS[precision], _stream(stream))
        self._check(st, "pt_apply_exchange")
        return out

    def apply_exchange_mixed(self, phi, sigma, tgt=None, out=None, *, cell, kernel=None, precision="fp64",
                             stream=None):
        """out_j = -sum_ik sigma_ik phi_i IFFT[K FFT[conj(phi_k) tgt_j]] by the undiagonalised triple loop
        (N*N*M pair FFTs; tgt None: tgt = phi).  Returns (out, pair_ffts)."""
        self._orb(phi, precision, "phi")
        if tgt is not None:
            self._orb(tgt, precision, "tgt")
        _block(phi, cell, "phi")
        if tgt is not None:
            _block(tgt, cell, "tgt")
        if sigma.dtype != torch.complex128 or not sigma.is_contiguous() or sigma.device != self.device:
            raise ValueError("sigma must be a contiguous complex128 tensor on the device")
        _sized(sigma, phi.shape[0] ** 2, "sigma")
        ref = phi if tgt is None else tgt
        if out is None:
            out = torch.empty_like(ref)
        _result(out, ref.numel(), ref.dtype, self.device)
        g, k = _grid(cell), _kernel(kernel)
        n = C.c_longlong(0)
        st = self.lib.pt_apply_exchange_mixed(self.h, _ptr(phi), _ptr(sigma), phi.shape[0],
                                              None if tgt is None else _ptr(tgt), ref.shape[0], _ptr(out),
                                              C.byref(g), C.byref(k), L.PRECISIONS[precision], C.byref(n),
                                              _stream(stream))
        self._check(st, "pt_apply_exchange_mixed")
        return out, int(n.value)

    def apply_exchange_batched(self, items, *, precision="fp32", stream=None):
        """Batched V_x applications.  items: list of dicts with keys src, occ, cell and optional
        tgt, out, kernel (as apply_exchange).  Returns (outs, pair_ffts, graph_nodes)."""
        arr = (L.pt_exchange_item * len(items))()
        outs, keep = [], []
        for k, it in enumerate(items):
            src = self._orb(it["src"], precision, "src")
            tgt = it.get("tgt")
            if tgt is not None:
                self._orb(tgt, precision, "tgt")
            occ = it["occ"].to(device=self.device, dtype=torch.float64).contiguous()
            ref = src if tgt is None else tgt
            where = f"item {k}: "
            _block(src, it["cell"], "src", where)
            if tgt is not None:
                _block(tgt, it["cell"], "tgt", where)
            if occ.numel() < src.shape[0]:
                raise PtimError(L.PT_INVALID_ARG, f"{where}occ holds {occ.numel()} occupations for {src.shape[0]} orbitals")
            out = it.get("out")
            if out is None:
                out = torch.empty_like(ref)
            _result(out, ref.numel(), ref.dtype, self.device, where=where)
            keep.append(occ)
            outs.append(out)
            a = arr[k]
            a.src, a.occ, a.N = src.data_ptr(), occ.data_ptr(), src.shape[0]
            a.tgt, a.M = (None, 0) if tgt is None else (tgt.data_ptr(), tgt.shape[0])
            a.out = out.data_ptr()
            a.grid, a.kernel = _grid(it["cell"]), _kernel(it.get("kernel"))
        pairs, nodes = C.c_longlong(0), C.c_size_t(0)
        st = self.lib.pt_apply_exchange_batched(self.h, arr, len(items), L.PRECISIONS[precision], C.byref(pairs),
                                                C.byref(nodes), _stream(stream))
        self._check(st, "pt_apply_exchange_batched")
        return outs, int(pairs.value), int(nodes.value)

    # ---- ACE --------------------------------------------------------------------------------
    def build_ace(self, phi, occ, *, cell, kernel=None, precision="fp64", stream=None) -> Ace:
        self._orb(phi, precision, "phi")
        _block(phi, cell, "phi")
        occ = occ.to(device=self.device, dtype=torch.float64).contiguous()
        if occ.numel() < phi.shape[0]:
            raise PtimError(L.PT_INVALID_ARG, f"occ holds {occ.numel()} occupations for {phi.shape[0]} orbitals")
        g, k = _grid(cell), _kernel(kernel)
        h = C.c_void_p()
        st = self.lib.pt_build_ace(self.h, _ptr(phi), _ptr(occ), phi.shape[0], C.byref(g), C.byref(k),
                                   L.PRECISIONS[precision], C.byref(h), _stream(stream))
        self._check(st, "pt_build_ace")
        return Ace(self, h, phi.shape[0], cell, precision)

    def build_ace_from(self, W, phi, *, cell, precision="fp64", stream=None) -> Ace:
        self._orb(W, precision, "W")
        self._orb(phi, precision, "phi")
        _block(phi, cell, "phi")
        _sized(W, phi.numel(), "W")
        g = _grid(cell)
        h = C.c_void_p()
        st = self.lib.pt_build_ace_from(self.h, _ptr(W), _ptr(phi), phi.shape[0], C.byref(g),
                                        L.PRECISIONS[precision], C.byref(h), _stream(stream))
        self._check(st, "pt_build_ace_from")
        return Ace(self, h, phi.shape[0], cell, precision)

    def apply_ace(self, ace: Ace, psi, out=None, stream=None):
        self._orb(psi, ace.precision, "psi")
        _block(psi, ace.cell, "psi")
        if out is None:
            out = torch.empty_like(psi)
        _result(out, psi.numel(), psi.dtype, self.device)
        st = self.lib.pt_apply_ace(self.h, ace.handle, _ptr(psi), psi.shape[0], _ptr(out), _stream(stream))
        self._check(st, "pt_apply_ace")
        return out

    # ---- overlaps ---------------------------------------------------------------------------
    def overlap(self, A, B=None, *, cell, precision="fp64", out=None, stream=None):
        """C[i][j] = dV <A_i|B_j> as an (N1, N2) complex128 device tensor (B None: B = A)."""
        self._orb(A, precision, "A")
        B = A if B is None else B
        self._orb(B, precision, "B")
        _block(A, cell, "A")
        _block(B, cell, "B")
        if out is None:
            out = torch.empty((A.shape[0], B.shape[0]), dtype=torch.complex128, device=self.device)
        _result(out, A.shape[0] * B.shape[0], torch.complex128, self.device)
        g = _grid(cell)
        st = self.lib.pt_overlap(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], C.byref(g),
                                 L.PRECISIONS[precision], _ptr(out), _stream(stream))
        self._check(st, "pt_overlap")
        return out

    def rotate(self, A, B, *, cell, precision="fp64", out=None, stream=None):
        """out_j = sum_k B[k, j] A_k for an (N1, N2) complex128 device matrix B."""
        self._orb(A, precision, "A")
        B = B.to(device=self.device, dtype=torch.complex128).contiguous()
        if B.dim() != 2 or B.shape[0] != A.shape[0]:
            raise ValueError("B must be (N1, N2) with N1 = A.shape[0]")
        _block(A, cell, "A")
        if out is None:
            out = torch.empty((B.shape[1],) + tuple(A.shape[1:]), dtype=A.dtype, device=self.device)
        _result(out, B.shape[1] * _points(cell), A.dtype, self.device)
        g = _grid(cell)
        st = self.lib.pt_rotate(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[1], C.byref(g),
                                L.PRECISIONS[precision], _ptr(out), _stream(stream))
        self._check(st, "pt_rotate")
        return out

    # ---- Hamiltonian ------------------------------------------------------------------------
    def apply_H(self, psi, vloc, ace: Ace | None = None, alpha=0.25, ecut=10.0, *, cell, precision="fp64",
                A=None, out=None, stream=None):
        """H psi with the velocity-gauge vector potential A (3 floats, or None for no field)."""
        self._orb(psi, precision, "psi")
        _block(psi, cell, "psi")
        vloc = vloc.to(device=self.device, dtype=torch.float64).contiguous()
        _sized(vloc, _points(cell), "vloc")
        if out is None:
            out = torch.empty_like(psi)
        _result(out, psi.numel(), psi.dtype, self.device)
        g = _grid(cell)
        st = self.lib.pt_apply_H(self.h, _ptr(psi), psi.shape[0], _ptr(out), _ptr(vloc),
                                 None if ace is None else ace.handle, float(alpha), float(ecut), _vec3(A),
                                 C.byref(g), L.PRECISIONS[precision], _stream(stream))
        self._check(st, "pt_apply_H")
        return out

    def current(self, phi, sigma, *, cell, precision="fp64", A=None, spin=2.0, stream=None):
        """J = spin/Omega Re Tr[P (-i grad + A)] as a (3,) numpy array (synchronises the stream)."""
        self._orb(phi, precision, "phi")
        _block(phi, cell, "phi")
        sigma = sigma.to(device=self.device, dtype=torch.complex128).contiguous()
        _sized(sigma, phi.shape[0] ** 2, "sigma")
        g = _grid(cell)
        J = (C.c_double * 3)()
        st = self.lib.pt_current(self.h, _ptr(phi), _ptr(sigma), phi.shape[0], C.byref(g), L.PRECISIONS[precision],
                                 _vec3(A), float(spin), J, _stream(stream))
        self._check(st, "pt_current")
        return np.array([J[0], J[1], J[2]])

    # ---- self-consistent local potential ------------------------------------------------------
    def density(self, phi, sigma, *, cell, precision="fp64", spin=2.0, out=None, stream=None):
        """rho = spin * P(r, r), P = Phi sigma Phi^* (float64 tensor shaped like one orbital)."""
        self._orb(phi, precision, "phi")
        _block(phi, cell, "phi")
        sigma = sigma.to(device=self.device, dtype=torch.complex128).contiguous()
        _sized(sigma, phi.shape[0] ** 2, "sigma")
        if out is None:
            out = torch.empty(phi.shape[1:], dtype=torch.float64, device=self.device)
        _result(out, _points(cell), torch.float64, self.device)
        g = _grid(cell)
        st = self.lib.pt_density(self.h, _ptr(phi), _ptr(sigma), phi.shape[0], C.byref(g), L.PRECISIONS[precision],
                                 float(spin), _ptr(out), _stream(stream))
        self._check(st, "pt_density")
        return out

    def hxc_potential(self, rho, vloc=None, *, cell, energies=False, out=None, stream=None):
        """vloc + V_H[rho] + v_xc(rho) (FP64); with energies=True also returns (E_H, E_xc)."""
        rho = rho.to(device=self.device, dtype=torch.float64).contiguous()
        _sized(rho, _points(cell), "rho")
        if vloc is not None:
            vloc = vloc.to(device=self.device, dtype=torch.float64).contiguous()
            _sized(vloc, _points(cell), "vloc")
        if out is None:
            out = torch.empty_like(rho)
        _result(out, rho.numel(), torch.float64, self.device)
        g = _grid(cell)
        e = (C.c_double * 2)()
        st = self.lib.pt_hxc_potential(self.h, _ptr(rho), None if vloc is None else _ptr(vloc), C.byref(g),
                                       _ptr(out), e if energies else None, _stream(stream))
        self._check(st, "pt_hxc_potential")
        return (out, (float(e[0]), float(e[1]))) if energies else out

    # ---- occupations ----------------------------------------------------------------------
    def diag_occupations(self, sigma, stream=None):
        sigma = sigma.to(device=self.device, dtype=torch.complex128).contiguous()
        if sigma.dim() != 2 or sigma.shape[0] != sigma.shape[1]:
            raise PtimError(L.PT_INVALID_ARG, "sigma must be a square (N, N) matrix")
        N = sigma.shape[0]
        Q = torch.empty_like(sigma)
        d = torch.empty(N, dtype=torch.float64, device=self.device)
        st = self.lib.pt_diag_occupations(self.h, _ptr(sigma), N, _ptr(Q), _ptr(d), _stream(stream))
        self._check(st, "pt_diag_occupations")
        return Q, d

    # ---- PT-IM step -------------------------------------------------------------------------
    def ptim_step(self, phi, sigma, vloc, *, cell, kernel=None, precision="fp64", dt=0.5, alpha=0.25, ecut=10.0,
                  tol=1e-6, max_outer=30, max_inner=200, anderson_depth=20, anderson_beta=1.0, use_ace=True,
                  spin=2.0, hxc=False, A=None, stream=None, allow_unconverged=False):
        """Advance (phi, sigma) by one PT-IM(-ACE) step in place; returns the step statistics."""
        self._orb(phi, precision, "phi")
        if sigma.dtype != torch.complex128 or not sigma.is_contiguous() or sigma.device != self.device:
            raise ValueError("sigma must be a contiguous complex128 tensor on the device")
        _block(phi, cell, "phi")
        _sized(sigma, phi.shape[0] ** 2, "sigma")
        vloc = vloc.to(device=self.device, dtype=torch.float64).contiguous()
        _sized(vloc, _points(cell), "vloc")
        p = L.pt_ptim_params(dt, alpha, ecut, tol, max_outer, max_inner, anderson_depth, anderson_beta,
                             int(bool(use_ace)), spin, int(bool(hxc)),
                             (C.c_double * 3)(*(A if A is not None else (0.0, 0.0, 0.0))))
        s = L.pt_ptim_stats()
        g, k = _grid(cell), _kernel(kernel)
        st = self.lib.pt_ptim_step(self.h, _ptr(phi), _ptr(sigma), phi.shape[0], _ptr(vloc), C.byref(g), C.byref(k),
                                   C.byref(p), L.PRECISIONS[precision], C.byref(s), _stream(stream))
        if not (st == L.PT_OK or (allow_unconverged and st == L.PT_NOT_CONVERGED)):
            self._check(st, "pt_ptim_step")
        return {"status": L.STATUS_NAMES[st], "outer": s.outer, "inner": s.inner, "residual": s.residual,
                "exch_energy": s.exch_energy, "orth_error": s.orth_error, "converged": bool(s.converged),
                "pair_ffts": int(s.pair_ffts), "exchange_calls": int(s.exchange_calls),
                "exchange_ms": float(s.exchange_ms), "eig_sweeps": int(s.eig_sweeps),
                "total_energy": float(s.total_energy), "pure_state": bool(s.pure_state), "ace_warm": bool(s.ace_warm),
                "pass_inner": [int(s.pass_inner[i]) for i in range(min(int(s.passes), 16))],
                "sinv_path": [int(s.sinv_path[i]) for i in range(4)], "s_dev_max": float(s.s_dev_max),
                "sinv_mixed_fallback": bool(s.sinv_mixed_fallback),
                "plane_waves": int(s.plane_waves),
                "phase_ms": {n: float(s.phase_ms[i]) for i, n in enumerate(L.PHASES)}}


def ptim_footprint(N: int, cell, precision: str = "fp32", anderson_depth: int = 20) -> int:
    """Upper bound of the device bytes one PT-IM step of this size makes a fresh context allocate."""
    g = _grid(cell)
    return int(L.load().pt_ptim_footprint(int(N), C.byref(g), L.PRECISIONS[precision], int(anderson_depth)))


def kernel_launches() -> int:
    return int(L.load().pt_kernel_launches())
