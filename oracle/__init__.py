"""FP64 CPU oracle for L-JSDE / RL-JSDE (test infrastructure).

This package is the plain, slow reference that the CUDA library is checked
against.  Only the test suite, the package smoke check and the CPU-baseline
leg of the benchmark may import it; the library never does, and the two share
no code.  The arithmetic lives in ``ljsde_oracle.c`` (direct L-JSDE of
Sec. IV / Eqs. 4-10, recurrent RL-JSDE of Eqs. 11-17, the sensor of Eq. 1);
this module only marshals numpy arrays into it.

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):

* ``measure``            -- pinned: hand-evaluated sums, linearity; the
  aperture layout against the three-quarter codes it generalises.
* ``window_solve``       -- pinned: brute-force weighted least squares per
  candidate on tiny windows, energy identity, single-atom recovery,
  identity-measurement reduction to ``numpy.fft.fft2`` with exact sparse
  recovery, measurement consistency, invariances.
* ``window_tables``      -- pinned: dense ``M^H diag(w) M`` built with
  ``numpy.exp``, Hermitian symmetry, Cauchy-Schwarz bound.
* ``reconstruct``        -- pinned through the above plus direct == recurrent;
  aperture layouts: three-quarter apertures == opaque codes, quarter
  sampling and the full 2x2 aperture reduce to closed forms built on
  ``numpy.fft.fft2``, unobservable Nyquist candidates never selected.
* ``pairs=1`` (conjugate-pair update, a variant of the paper's loop) --
  pinned: residual and model stay exactly real, E_w non-increasing for
  gamma <= 1, identity measurement recovers conjugate-pair sparse signals
  exactly and equals two single updates per pair, direct == recurrent.
* ``frequency_weight``   -- parity unpinned: default q, its form and its square.
  The paper gives no formula (Sec. IV, Eq. 11 says only that q favours low
  frequencies); the tests check the stated reading's properties (1 at DC,
  symmetric, isotropic, non-increasing in |k|, zero only at (W/2, W/2)),
  which the same reading without the square would pass too.  No parity
  check depends on it: the GPU tests also run q = 1 and user tables.
* spatial weight ``w_m = rho^d_m`` (inside ``reconstruct``) -- parity
  unpinned: w_m functional form.  The paper (Sec. III, Eq. 8) only calls the
  weight isotropic and decaying from the window centre; the mirror/transpose
  test pins its centring on the target block, not its form (rho^(d^2) would
  pass it).
* binary32 rounding of the argmax (reading of Eqs. 10-11, Table I's
  complex64 tables) -- pinned: two scores 2^-40 apart tie after rounding and
  go to the lower index, 2^-20 apart they do not.
* ``count_local_masks``  -- pinned: Table I (64 local masks for a 32-pixel
  period) and closed-form counts for small tiles.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["Params", "LAYOUT_THREE_QUARTER", "LAYOUT_APERTURE", "measure", "window_solve", "window_tables", "reconstruct",
           "count_local_masks", "frequency_weight", "load"]

_lib = None


class _CParams(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("block", ctypes.c_int), ("nu_max", ctypes.c_int),
                ("gamma_odc", ctypes.c_double), ("rho_decay", ctypes.c_double),
                ("q_mode", ctypes.c_int), ("q_table", ctypes.POINTER(ctypes.c_double)),
                ("layout", ctypes.c_int), ("pairs", ctypes.c_int)]


LAYOUT_THREE_QUARTER = 0   # mask code = index 2 * dy + dx of the opaque sub-pixel
LAYOUT_APERTURE = 1        # mask code = bit set of the transparent sub-pixels


class Params:
    """Reconstruction parameters (window W, block B, nu_max, gamma_odc, rho, q,
    the meaning of the mask codes, and the update: one complex coefficient
    per iteration, or ``pairs=1`` for the conjugate-pair update)."""

    def __init__(self, window=32, block=4, nu_max=100, gamma_odc=0.5, rho_decay=0.7,
                 q_mode=0, q_table=None, layout=LAYOUT_THREE_QUARTER, pairs=0):
        self.window, self.block, self.nu_max = int(window), int(block), int(nu_max)
        self.gamma_odc, self.rho_decay, self.q_mode = float(gamma_odc), float(rho_decay), int(q_mode)
        self.q_table = None if q_table is None else np.ascontiguousarray(q_table, dtype=np.float64)
        self.layout = int(layout)
        self.pairs = int(pairs)

    def c(self):
        qp = None
        if self.q_table is not None:
            qp = self.q_table.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return _CParams(self.window, self.block, self.nu_max, self.gamma_odc, self.rho_decay,
                        self.q_mode, qp, self.layout, self.pairs)


def load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(st, what):
    if st != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, st))


def measure(f: np.ndarray, mask: np.ndarray, layout: int = LAYOUT_THREE_QUARTER) -> np.ndarray:
    """Eq. 1 measurement: each L-pixel sums its transparent sub-pixels (three
    for three-quarter sampling; the code's bit set for ``LAYOUT_APERTURE``)."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    lr_h, lr_w = mask.shape
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (2 * lr_h, 2 * lr_w)
    y = np.empty((lr_h, lr_w), np.float64)
    _check(load().orc_measure(_p(f), _p(mask), lr_h, lr_w, int(layout), _p(y)), "measure")
    return y


def _window_arrays(pixels):
    nm = len(pixels)
    npx = np.zeros(max(nm, 1), np.int32)
    eta = np.zeros(4 * max(nm, 1), np.int32)
    gam = np.zeros(4 * max(nm, 1), np.int32)
    for m, px in enumerate(pixels):
        assert 1 <= len(px) <= 4
        npx[m] = len(px)
        for i, (e, g) in enumerate(px):
            eta[4 * m + i], gam[4 * m + i] = e, g
    return nm, npx, eta, gam


def window_solve(pixels, w, y, params: Params, recurrent=False):
    """Run the greedy loop on one model window with explicit measurements.

    ``pixels[m]`` lists the (eta, gamma) window coordinates integrated by
    measurement m; ``w`` are the spatial weights and ``y`` the (real or
    complex) measured values.  Returns a dict with the coefficients ``c``
    (W x W complex), ``sel``, ``dc`` (gamma_odc * delta, complex),
    ``gap``, and, for the direct variant, ``energy`` (nu_max + 1) and the
    final residual ``r``.
    """
    W, nu = params.window, params.nu_max
    nm, npx, eta, gam = _window_arrays(pixels)
    w = np.ascontiguousarray(w, dtype=np.float64)
    y = np.asarray(y)
    y_re = np.ascontiguousarray(y.real, dtype=np.float64)
    y_im = np.ascontiguousarray(y.imag, dtype=np.float64) if np.iscomplexobj(y) else None
    c = np.zeros(W * W * 2)
    sel = np.zeros(max(nu, 1), np.int32)
    dc = np.zeros(2 * max(nu, 1))
    gap = np.zeros(max(nu, 1))
    energy = np.zeros(nu + 1)
    r = np.zeros(2 * max(nm, 1))
    pc = params.c()
    st = load().orc_window_solve(int(recurrent), W, nm, _p(npx), _p(eta), _p(gam), _p(w), _p(y_re),
                                 _p(y_im), ctypes.byref(pc), _p(c), _p(sel), _p(dc), _p(gap),
                                 None if recurrent else _p(energy), None if recurrent else _p(r))
    _check(st, "window_solve")
    out = dict(c=(c[0::2] + 1j * c[1::2]).reshape(W, W), sel=sel[:nu].copy(),
               dc=dc[0:2 * nu:2] + 1j * dc[1:2 * nu:2], gap=gap[:nu].copy())
    if not recurrent:
        out["energy"] = energy
        out["r"] = r[0:2 * nm:2] + 1j * r[1:2 * nm:2]
    return out


def window_tables(pixels, w, W):
    """B (nm x W^2), C (W^2 x W^2) and D (W^2) of Eqs. 12-14 for one window."""
    nm, npx, eta, gam = _window_arrays(pixels)
    K = W * W
    w = np.ascontiguousarray(w, dtype=np.float64)
    B = np.zeros(2 * max(nm, 1) * K)
    C = np.zeros(2 * K * K)
    D = np.zeros(K)
    _check(load().orc_window_tables(W, nm, _p(npx), _p(eta), _p(gam), _p(w), _p(B), _p(C), _p(D)),
           "window_tables")
    B = (B[0::2] + 1j * B[1::2])[: nm * K].reshape(nm, K)
    C = (C[0::2] + 1j * C[1::2]).reshape(K, K)
    return B, C, D


def reconstruct(y, mask, params: Params, blocks=None, recurrent=False, n_threads=None,
                trace=False):
    """Reconstruct an image measured by Eq. 1 (or a list of its blocks).

    ``y`` are the lr_h x lr_w measurements, ``mask`` the per-pixel codes in
    ``params.layout`` (opaque sub-pixel 0..3, or transparent set 0..15).  ``blocks`` lists linear block indices ``bi * (2 lr_w / B) + bj``
    (default: every block); only those blocks of the returned HR image are
    written (the rest stay NaN).  With ``trace`` the per-block selection
    sequence, coefficient increments and FP64 score gaps are returned too.
    """
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    lr_h, lr_w = mask.shape
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert y.shape == mask.shape
    hr = np.full((2 * lr_h, 2 * lr_w), np.nan)
    nb_total = (2 * lr_h // params.block) * (2 * lr_w // params.block)
    bl = None if blocks is None else np.ascontiguousarray(blocks, dtype=np.int32)
    n = nb_total if bl is None else len(bl)
    nu = params.nu_max
    sel = np.zeros((max(n, 1), max(nu, 1)), np.int32) if trace else None
    dc = np.zeros((max(n, 1), 2 * max(nu, 1))) if trace else None
    gap = np.zeros((max(n, 1), max(nu, 1))) if trace else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    pc = params.c()
    st = load().orc_reconstruct(int(recurrent), _p(y), _p(mask), lr_h, lr_w, ctypes.byref(pc),
                                _p(bl), n, _p(hr), _p(sel), _p(dc), _p(gap), int(n_threads))
    _check(st, "reconstruct")
    if not trace:
        return hr
    return hr, dict(sel=sel[:n, :nu], dc=dc[:n, 0:2 * nu:2] + 1j * dc[:n, 1:2 * nu:2],
                    gap=gap[:n, :nu])


def frequency_weight(params: Params) -> np.ndarray:
    """The W x W frequency weight q of Eq. 11 that the loop uses."""
    W = params.window
    q = np.zeros(W * W)
    pc = params.c()
    _check(load().orc_frequency_weight(ctypes.byref(pc), _p(q)), "frequency_weight")
    return q.reshape(W, W)


def count_local_masks(mask, params: Params):
    """(all, interior) number of distinct local measurement matrices."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    a, b = ctypes.c_int(), ctypes.c_int()
    pc = params.c()
    _check(load().orc_count_local_masks(_p(mask), mask.shape[0], mask.shape[1], ctypes.byref(pc),
                                        ctypes.byref(a), ctypes.byref(b)), "count_local_masks")
    return a.value, b.value
