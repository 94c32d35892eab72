"""Helpers for the GPU parity tests: a handle wrapper around the C ABI and
natural-layout conversions.  Inputs come from ``inputs`` (seeded); expected
values come from ``oracle`` only."""
from __future__ import annotations

import numpy as np

import paper_1611_01034_gb300 as tm

try:
    import torch
except ImportError:  # pragma: no cover
    torch = None


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t) -> np.ndarray:
    return t.cpu().numpy()


def rel(a, b) -> float:
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


class GPU:
    """One handle bound to torch's current stream, with the gauge field loaded."""

    def __init__(self, U: np.ndarray, **kw):
        self.L = tuple(U.shape[:4])
        kw.setdefault("L", self.L)
        self.p = tm.params(**kw)
        self.stream = torch.cuda.current_stream()
        self.h = tm.tm_create(self.p, self.stream)
        tm.tm_load_gauge(self.h, dev(U))
        self.nv = self.p.nv
        self.Lc = tuple(self.L[d] // self.p.agg[d] for d in range(4))

    def close(self):
        if self.h is not None:
            tm.tm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- fields --------------------------------------------------------------
    def field(self, level: int, prec: int, nrhs: int = 1):
        n = tm.tm_field_bytes(self.h, level, prec, nrhs)
        return torch.zeros(n, dtype=torch.uint8, device="cuda")

    def pack(self, level: int, prec: int, a: np.ndarray, nrhs: int = 1):
        f = self.field(level, prec, nrhs)
        tm.tm_pack(self.h, level, prec, dev(a.astype(np.complex128)), f, nrhs)
        return f

    def unpack(self, level: int, prec: int, f, shape, nrhs: int = 1) -> np.ndarray:
        out = torch.zeros(int(np.prod(shape)), dtype=torch.complex128, device="cuda")
        tm.tm_unpack(self.h, level, prec, f, out, nrhs)
        torch.cuda.synchronize()
        return host(out).reshape(shape)

    def fine_shape(self, nrhs=None):
        return self.L + (4, 3) if nrhs is None else (nrhs,) + self.L + (4, 3)

    def coarse_shape(self, nrhs=None):
        s = self.Lc + (2 * self.nv,)
        return s if nrhs is None else (nrhs,) + s

    # -- operations ---------------------------------------------------------------
    def apply_fine(self, psi: np.ndarray, prec: int, nrhs: int = 1) -> np.ndarray:
        fi = self.pack(0, prec, psi, nrhs)
        fo = self.field(0, prec, nrhs)
        tm.tm_apply(self.h, 0, prec, fi, fo, nrhs)
        return self.unpack(0, prec, fo, psi.shape, nrhs)

    def sap(self, b, x0, sweeps: int, prec: int) -> np.ndarray:
        fb = self.pack(0, prec, b) if b is not None else None
        fx = self.pack(0, prec, x0)
        tm.tm_sap(self.h, prec, fb, fx, sweeps, 1)
        return self.unpack(0, prec, fx, x0.shape)

    def export(self, what: int, shape) -> np.ndarray:
        out = np.zeros(int(np.prod(shape)), dtype=np.complex128)
        tm.tm_export(self.h, what, out, out.nbytes)
        return out.reshape(shape)

    def P_columns(self) -> np.ndarray:
        return self.export(tm.TM_EXPORT_P, (2 * self.nv,) + self.L + (4, 3))

    def Dc_blocks(self) -> np.ndarray:
        n = 2 * self.nv
        return self.export(tm.TM_EXPORT_DC, self.Lc + (9, n, n))

    def clover(self) -> np.ndarray:
        return self.export(tm.TM_EXPORT_CLOVER, self.L + (2, 6, 6))
