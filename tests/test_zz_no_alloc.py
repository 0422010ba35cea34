"""mcd_connections_noalloc: the connection dump for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).
Collected last on purpose.  It must give the same entries as mcd_connections,
call after call, and refuse bases larger than its fixed scratch."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from workloads import configs as C

from gpu_common import device_ctx

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


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


def test_noalloc_rejects_bases_above_its_scratch():
    pkg.build()
    w = C.tilted12_u8()
    ctx = device_ctx(w, nf=(1 << 18) + 1)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_connections_noalloc()
    assert e.value.status == -1 and "262144" in str(e.value)
