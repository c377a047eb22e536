"""Build and load the CUDA library (libshf.so) in-tree.

The library is compiled with nvcc for sm_103a only, one translation unit per
source file, in parallel, into ``paper_0710_5912_gb300/lib/libshf.so``.  Nothing
is installed into site-packages.  If the library is missing or stale and cannot
be built, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
ROOT_DIR = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(ROOT_DIR, "include")
BUILD_DIR = os.path.join(PKG_DIR, "_build")
LIB_DIR = os.path.join(PKG_DIR, "lib")
LIB_PATH = os.path.join(LIB_DIR, "libshf.so")

SOURCES = ["step_kernels.cu", "step_rows.cu", "step_cols.cu", "diag_kernels.cu", "shf_api.cu", "mass_static.cu", "peaks.cu"]
HEADERS = ["fft_block.cuh", "shf_internal.cuh", "step_common.cuh"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr"]

_lock = threading.Lock()
_lib = None


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libshf")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, s) for s in _sources()] + [os.path.join(CSRC, h) for h in HEADERS]
    files.append(os.path.join(INCLUDE, "shf.h"))
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def is_stale() -> bool:
    return not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < _inputs_mtime()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu source for sm_103a and link libshf.so; returns its path."""
    with _lock:
        if not force and not is_stale():
            return LIB_PATH
        nvcc = nvcc_path()
        os.makedirs(BUILD_DIR, exist_ok=True)
        os.makedirs(LIB_DIR, exist_ok=True)
        procs = []
        objs = []
        for src in _sources():
            obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-c",
                   os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        errors = []
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                errors.append(f"--- {src} ---\n{out.decode(errors='replace')}")
            elif verbose and out:
                print(out.decode(errors="replace"), flush=True)
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        tmp = LIB_PATH + ".tmp"
        link = [nvcc, *ARCH_FLAGS, "-shared", "-o", tmp, *objs]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, LIB_PATH)
        return LIB_PATH


def load(auto_build: bool = True) -> ctypes.CDLL:
    """Load libshf.so (building it first if missing or stale and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    if is_stale():
        if not auto_build:
            raise RuntimeError(f"{LIB_PATH} is missing or stale; run __graft_entry__.build()")
        build()
    lib = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
    _declare(lib)
    _lib = lib
    return lib


c_int, c_double, c_int64, c_uint64, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_char_p)
P_double = ctypes.POINTER(ctypes.c_double)
P_float = ctypes.POINTER(ctypes.c_float)
P_int = ctypes.POINTER(ctypes.c_int)
P_int64 = ctypes.POINTER(ctypes.c_int64)
P_uint64 = ctypes.POINTER(ctypes.c_uint64)
P_void_p = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); mirrors include/shf.h
SIGNATURES = {
    "shf_version": (c_int, []),
    "shf_strerror": (c_char_p, [c_int]),
    "shf_last_error": (c_char_p, [c_void_p]),
    "shf_create_grid": (c_int, [P_void_p, c_int, c_int, c_double, c_int, c_int, c_void_p]),
    "shf_destroy_grid": (c_int, [c_void_p]),
    "shf_set_params": (c_int, [c_void_p, c_double, c_double, c_double, c_double, c_double, c_double,
                               c_double, c_double]),
    "shf_set_fields": (c_int, [c_void_p, P_double, P_double, P_double]),
    "shf_set_fields_f32": (c_int, [c_void_p, P_float, P_float, P_float]),
    "shf_get_fields_f32": (c_int, [c_void_p, P_float, P_float, P_float]),
    "shf_step_host_f32": (c_int, [c_void_p, c_int64, P_float, P_float, P_float, P_float, P_float, P_float]),
    "shf_init_noise": (c_int, [c_void_p, c_uint64, c_double]),
    "shf_bind_device_fields": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "shf_set_step": (c_int, [c_void_p, c_int64]),
    "shf_step": (c_int, [c_void_p, c_int64]),
    "shf_profile_step": (c_int, [c_void_p, c_int64, P_double, c_int]),
    "shf_sync": (c_int, [c_void_p]),
    "shf_get_fields": (c_int, [c_void_p, P_double, P_double, P_double]),
    "shf_get_time": (c_int, [c_void_p, P_int64, P_double, P_double, P_int64]),
    "shf_mass": (c_int, [c_void_p, P_double]),
    "shf_structure_factor": (c_int, [c_void_p, P_double, c_int, P_double]),
    "shf_gradient_tensor": (c_int, [c_void_p, P_double, P_double]),
    "shf_autotune": (c_int, [c_void_p, c_char_p, P_int, c_int]),
    "shf_save": (c_int, [c_void_p, c_char_p]),
    "shf_load": (c_int, [c_void_p, c_char_p]),
    "shf_create_ensemble": (c_int, [P_void_p, c_int, P_int, P_int, P_double, P_double, P_uint64, c_double,
                                    c_int, c_void_p]),
    "shf_ensemble_member": (c_int, [c_void_p, c_int, P_void_p]),
    "shf_strain": (c_int, [c_int64, c_double, c_double, c_int, c_int, P_double, P_int64]),
    "shf_noise_fill": (c_int, [P_double, c_int64, c_uint64, c_double]),
    "shf_mass_static": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, P_double]),
    "shf_fma_peak": (c_int, [c_int, c_int, P_double]),
}


def _declare(lib):
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
