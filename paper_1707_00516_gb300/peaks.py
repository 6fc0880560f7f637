"""Roofline denominators measured on the GPU in use (``probe/peaks.cu``).

``measure()`` times, each once after a warm-up launch:

* the tensor pipe: tcgen05 ``kind::f8f6f4`` (e4m3, M 128 x N 256 x K 32) and
  block-scaled ``kind::mxf4`` (e2m1 with unit ue8m0 scale factors, M 128 x
  N 224 and 256 x K 64), operands in shared memory, one CTA per SM;
* the integer pipes: POPC alone, LOP3 alone, the plain form's inner
  sequence (AND, POPC, one 3-input add per two words), and the same count
  by a carry-save (Harley-Seal) tree, in word pairs;
* the binary tensor-core path: ``mma.sync m16n8k256 b1 AND + POPC``.

Each rate is reported per second (CUDA events, at the clock the probe ran
at) and per SM clock (clock64 over the timed loop).  ``mma_check()`` runs one
stage of MMAs on given 0/+-1 operands and returns D, so the tests can compare
both operand encodings with an integer matmul.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

_D = ctypes.POINTER(ctypes.c_double)


def load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build.build_peaks())
            lib.fastid_peaks_mma.restype = ctypes.c_int
            lib.fastid_peaks_mma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _D, _D,
                                             _D]
            lib.fastid_peaks_alu.restype = ctypes.c_int
            lib.fastid_peaks_alu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
            lib.fastid_peaks_b1.restype = ctypes.c_int
            lib.fastid_peaks_b1.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
            _lib = lib
    return _lib


K_BYTES = 128  # bytes of K per operand row in one probe stage


def encode(vals: np.ndarray, f4: bool) -> np.ndarray:
    """Operand rows of 0/+1/-1 values as the MMA reads them: e4m3 bytes
    (0x00, 0x38, 0xB8; 128 per row) or e2m1 nibbles (0x0, 0x2, 0xA; 256 per
    row, element 2i in the low nibble of byte i)."""
    v = np.asarray(vals)
    if f4:
        nib = np.where(v > 0, 0x2, np.where(v < 0, 0xA, 0x0)).astype(np.uint8)
        return (nib[:, 0::2] | (nib[:, 1::2] << 4)).astype(np.uint8)
    return np.where(v > 0, 0x38, np.where(v < 0, 0xB8, 0x00)).astype(np.uint8)


def mma_check(f4: bool, n: int, a_vals: np.ndarray, b_vals: np.ndarray) -> np.ndarray:
    """D = A B^T from one stage of tcgen05 MMAs on one CTA.  a_vals [128][K],
    b_vals [n][K] with K = 128 (FP8) or 256 (FP4) values in {-1, 0, 1}."""
    lib = load()
    a = np.ascontiguousarray(encode(a_vals, f4))
    b = np.ascontiguousarray(encode(b_vals, f4))
    assert a.shape == (128, K_BYTES) and b.shape == (n, K_BYTES)
    d = np.zeros((128, n), dtype=np.float32)
    ms, clk, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.fastid_peaks_mma(int(f4), n, 1, 1, 1, 0, a.ctypes.data, b.ctypes.data, d.ctypes.data, ctypes.byref(ms),
                              ctypes.byref(clk), ctypes.byref(mhz))
    if rc != 0:
        raise RuntimeError(f"fastid_peaks_mma returned {rc}")
    return d


def _calibrated(run, target_ms: float, iters: int):
    """Run once to warm up and size, then once at about target_ms."""
    ms, *_ = run(iters)
    iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
    return run(iters) + (iters,)


def measure(target_ms: float = 40.0) -> dict:
    """Probe every denominator; returns a dict of rates (see module doc)."""
    lib = load()
    out = {}
    import torch
    n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

    def mma(f4, n, kmma, nst=1, sync=0):
        def run(iters):
            ms, clk, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            rc = lib.fastid_peaks_mma(int(f4), n, iters, 0, nst, sync, None, None, None, ctypes.byref(ms),
                                      ctypes.byref(clk), ctypes.byref(mhz))
            if rc != 0:
                raise RuntimeError(f"fastid_peaks_mma({f4}, {n}) returned {rc}")
            return ms.value, clk.value, mhz.value
        ms, clk, mhz, iters = _calibrated(run, target_ms, 2000)
        flops_cta = 2.0 * 128 * n * kmma * 4 * iters
        return {"tflops": flops_cta * n_sms / (ms / 1e3) / 1e12, "flops_per_clk_sm": flops_cta / clk,
                "sm_mhz": mhz, "ms": ms, "shape": f"M128xN{n}xK{kmma}", "stages": nst, "sync": sync}

    out["fp8_f8f6f4"] = mma(False, 256, 32)
    out["fp4_mxf4_n224"] = mma(True, 224, 64)
    out["fp4_mxf4_n256"] = mma(True, 256, 64)
    # the operands cycled through four stages of shared memory, as the
    # comparison kernel's pipeline holds them
    out["fp8_f8f6f4_4stages"] = mma(False, 256, 32, 4)
    out["fp4_mxf4_n224_4stages"] = mma(True, 224, 64, 4)
    # and with the per-stage barrier wait and commit of the kernel's MMA thread
    out["fp8_f8f6f4_4stages_sync"] = mma(False, 256, 32, 4, 7)
    out["fp4_mxf4_n224_4stages_sync"] = mma(True, 224, 64, 4, 7)

    def alu(op, name):
        def run(iters):
            ms, clk, mhz, el = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            rc = lib.fastid_peaks_alu(op, iters, 2, ctypes.byref(ms), ctypes.byref(clk), ctypes.byref(mhz),
                                      ctypes.byref(el))
            if rc != 0:
                raise RuntimeError(f"fastid_peaks_alu({op}) returned {rc}")
            return ms.value, clk.value, mhz.value, el.value
        ms, clk, mhz, el, iters = _calibrated(run, target_ms, 256)
        # per SM per clock over the whole launch (event time x measured SM
        # clock): two CTAs of 1024 threads a SM run at once only below 33
        # registers a thread (the carry-save probe holds more, so its CTAs run
        # one at a time, and one CTA's own clocks would count its SM twice)
        return {"per_s": el / (ms / 1e3), "per_clk_sm": el / n_sms / (ms * 1e3 * mhz), "sm_mhz": mhz, "ms": ms,
                "counts": name}

    out["popc"] = alu(0, "POPC")
    out["lop3"] = alu(1, "LOP3")
    out["and_popc_add"] = alu(2, "POPC in AND + POPC + IADD3/2")
    out["harley_seal"] = alu(3, "word pairs counted by AND + carry-save tree + POPC/8")
    out["carry_save8"] = alu(4, "word pairs counted by the plain kernel's step: 8 AND + 4 full adders + 4 POPC + adds")

    def b1():
        def run(iters):
            ms, clk, mhz, bm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            rc = lib.fastid_peaks_b1(iters, 4, ctypes.byref(ms), ctypes.byref(clk), ctypes.byref(mhz),
                                     ctypes.byref(bm))
            if rc != 0:
                raise RuntimeError(f"fastid_peaks_b1 returned {rc}")
            return ms.value, clk.value, mhz.value, bm.value
        ms, clk, mhz, bm, iters = _calibrated(run, target_ms, 256)
        return {"bit_macs_per_s": bm / (ms / 1e3), "bit_macs_per_clk_sm": bm / n_sms / (ms * 1e3 * mhz), "sm_mhz": mhz,
                "ms": ms}

    out["b1_and_popc"] = b1()
    out["sms"] = n_sms
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(measure(), indent=1))
