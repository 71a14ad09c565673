"""bspai_gmres_noalloc: the GMRES solve for callers that cannot allocate device
memory while they run -- a host program that handed the GPU's memory to its
own pool allocator up front, or code that must not call cudaMalloc/cudaFree
(which can synchronise the whole device) once it is running.

Checked through the C ABI against bspai_gmres, the allocating entry point.
Both run the same kernels in the same order, so the corrections must be
bit-identical: on two calls in a row, after a call on another system with a
larger kmax has left different contents (a longer Hessenberg matrix, more
reduction slots, another sequence count) in the shared fixed block.  A warm
call must also leave the device's stream-ordered memory pool and torch's
allocator where they were.  Kept in a file that pytest collects last."""
import ctypes
import os

import numpy as np
import pytest
import torch

from gpu_helpers import dev, gpu_bucket, gpu_build, host, lib
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_RESERVED_CURRENT, _USED_CURRENT, _USED_HIGH = 0x5, 0x7, 0x8  # cudaMemPoolAttr values


@pytest.fixture(scope="module")
def B():
    return lib()


def _cudart():
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    here = os.path.dirname(torch.__file__)
    for root, _, files in os.walk(os.path.join(os.path.dirname(here), "nvidia")):
        for f in files:
            if f.startswith("libcudart.so"):
                return ctypes.CDLL(os.path.join(root, f))
    pytest.skip("no libcudart to read the memory pool with")


class _Pool:
    """The current device's default stream-ordered memory pool (the one the
    library's allocating calls draw on), read through the CUDA runtime."""

    def __init__(self):
        self.rt = _cudart()
        d = ctypes.c_int()
        assert self.rt.cudaGetDevice(ctypes.byref(d)) == 0
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), d) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, _USED_HIGH, ctypes.byref(z)) == 0


def _system(B, grid, seed):
    wl = W.workload("convdiff3d", grid=grid)
    A, P = wl["A"], wl["pattern"]
    g = gpu_build(B, wl)
    bk = gpu_bucket(B, g["M"], P.nnz, 2.0 ** -16, wl["precs"])
    Ah = B.matrix_create(g["A"])
    r = dev(np.random.default_rng(seed).uniform(-1, 1, A.n) * np.abs(wl["b"]).max())
    return wl, bk, Ah, r


@pytest.mark.parametrize("ug", ["fp32", "fp64"])
def test_noalloc_matches_allocating_gmres_twice(B, ug):
    wl, bk, Ah, r = _system(B, 16, 11)
    n = wl["A"].n
    o = B.opts(tau=1e-6, kmax=200)
    d_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ref = B.gmres(Ah, bk["BM"], r, d_ref, ug, ug, o)
    dr = host(d_ref)
    # another system and a larger kmax first, so that the block holds stale data
    wl2, bk2, Ah2, r2 = _system(B, 12, 12)
    d2 = torch.empty(wl2["A"].n, dtype=torch.float64, device="cuda")
    other = B.gmres_noalloc(Ah2, bk2["BM"], r2, d2, ug, ug, B.opts(tau=1e-12, kmax=300))
    assert other["status"] == 0 and other["gmres_iters"][0] > ref["gmres_iters"][0]
    torch.cuda.synchronize()
    pool = _Pool()
    reserved0, used0 = pool.get(_RESERVED_CURRENT), pool.get(_USED_CURRENT)
    pool.reset_high()
    torch0 = torch.cuda.memory_allocated()
    for call in range(2):
        d = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        info = B.gmres_noalloc(Ah, bk["BM"], r, d, ug, ug, o)
        assert info["status"] == 0, (call, info)
        assert info["gmres_iters"] == ref["gmres_iters"], call
        assert info["relres"][0] == ref["relres"][0], call
        assert np.array_equal(host(d), dr), call
        del d
    torch.cuda.synchronize()
    assert pool.get(_USED_HIGH) == used0, "a no-allocation call drew on the memory pool"
    assert pool.get(_RESERVED_CURRENT) == reserved0
    assert torch.cuda.memory_allocated() == torch0


def test_noalloc_rejects_oversized_problem(B):
    wl, bk, Ah, r = _system(B, 64, 13)  # n = 262,144: a 300-step fp32 basis needs ~315 MB
    d = torch.zeros(wl["A"].n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.BspaiError) as e:
        B.gmres_noalloc(Ah, bk["BM"], r, d, "fp32", "fp32", B.opts(tau=1e-6, kmax=300))
    assert e.value.status == B.ERR_INVALID and "bytes of scratch" in str(e.value)
    assert torch.all(d == 0)
    # the same system with a basis that fits still runs
    info = B.gmres_noalloc(Ah, bk["BM"], r, d, "fp32", "fp32", B.opts(tau=1e-6, kmax=40))
    assert info["status"] == 0 and info["gmres_iters"][0] >= 1
