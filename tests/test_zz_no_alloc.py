"""mcd_connections_noalloc: the connection dump for callers that cannot
allocate device memory, such as an application that gives all device memory
to its own pool at start-up, or one under a fixed memory budget.  Its scratch
is a fixed array inside the library.  Collected last on purpose.  It must give
the same entries as mcd_connections, call after call, allocate nothing (the
device's default memory pool and its free memory stay as they were, while
mcd_connections draws on the pool), report the count when the capacity is too
small, and refuse bases larger than its fixed scratch."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from workloads import configs as C

from gpu_common import device_ctx

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# CUmemPool_attribute values (cuda.h)
RESERVED_MEM_HIGH, USED_MEM_CURRENT, USED_MEM_HIGH = 6, 7, 8


class DevicePool:
    """The default memory pool of device 0 and the device's free memory, read
    through the driver API (the pool that stream-ordered allocations use)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert self.cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        for attr in (RESERVED_MEM_HIGH, USED_MEM_HIGH):   # 0 resets the mark to the current value
            z = ctypes.c_uint64(0)
            assert self.cu.cuMemPoolSetAttribute(self.pool, attr, ctypes.byref(z)) == 0

    def free_bytes(self):
        free, total = ctypes.c_size_t(0), ctypes.c_size_t(0)
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        return free.value


def triples(ctx, fn):
    nnz = fn()
    rows = torch.empty(nnz, dtype=torch.int64, device=DEV)
    cols = torch.empty(nnz, dtype=torch.int64, device=DEV)
    vals = torch.empty(nnz, dtype=torch.float64, device=DEV)
    assert fn(rows, cols, vals) == nnz
    r, c, v = rows.cpu().numpy(), cols.cpu().numpy(), vals.cpu().numpy()
    assert np.all(np.diff(r) >= 0)            # grouped by row
    o = np.lexsort((c, r))
    return r[o], c[o], v[o]


@pytest.mark.parametrize("name,nf", [("ring8", 2000), ("tilted12", 1 << 18)])
def test_noalloc_matches_connections_twice(name, nf):
    pkg.build()
    w = C.WORKLOADS[name]()
    ctx = device_ctx(w, nf=nf)
    ref = triples(ctx, ctx.mcd_connections)
    for _ in range(2):
        got = triples(ctx, ctx.mcd_connections_noalloc)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_noalloc_allocates_nothing():
    pkg.build()
    w = C.tilted12_u8()
    ctx = device_ctx(w, nf=1 << 16)
    nnz = ctx.mcd_connections_noalloc()             # first call on the device: address look-up
    bufs = [torch.empty(nnz, dtype=dt, device=DEV) for dt in (torch.int64, torch.int64, torch.float64)]
    ctx.mcd_connections_noalloc(*bufs)
    torch.cuda.synchronize()
    pool = DevicePool()
    pool.reset_high()
    used0, free0 = pool.get(USED_MEM_CURRENT), pool.free_bytes()
    assert ctx.mcd_connections_noalloc() == nnz
    assert ctx.mcd_connections_noalloc(*bufs) == nnz
    torch.cuda.synchronize()
    assert pool.get(USED_MEM_HIGH) == used0          # no stream-ordered allocation, even briefly
    assert pool.free_bytes() >= free0                # no other device allocation
    # contrast: the allocating counterpart draws on the same pool during its call
    pool.reset_high()
    assert ctx.mcd_connections(*bufs) == nnz
    torch.cuda.synchronize()
    assert pool.get(USED_MEM_HIGH) > used0


def test_noalloc_capacity_too_small_reports_count():
    pkg.build()
    w = C.ring8_u4()
    ctx = device_ctx(w, nf=2000)
    nnz = ctx.mcd_connections_noalloc()
    bufs = [torch.empty(nnz - 1, dtype=dt, device=DEV) for dt in (torch.int64, torch.int64, torch.float64)]
    n = ctypes.c_int64(-7)
    ctx._sync_stream()
    st = ctx.L.mcd_connections_noalloc(ctx.h, *(ctypes.c_void_p(b.data_ptr()) for b in bufs), nnz - 1,
                                       ctypes.byref(n))
    assert st == -1 and n.value == nnz
    assert "capacity" in ctx.L.mcd_last_error(ctx.h).decode()


def test_noalloc_rejects_bases_above_its_scratch():
    pkg.build()
    w = C.tilted12_u8()
    ctx = device_ctx(w, nf=(1 << 18) + 1)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_connections_noalloc()
    assert e.value.status == -1 and "262144" in str(e.value)
