"""qfs_heights_noalloc: the allocation-free entry point gives the same heights as qfs_heights.

Some callers cannot allocate device memory when they call (inside a global-mode stream capture cudaMalloc is an
illegal call; under a framework allocator that owns the device there is nothing left to take).  For them the
library keeps one fixed scratch array on each device.  This file runs last so that a failure here leaves every
other test already run.
"""
import numpy as np
import pytest
import torch

from paper_2502_12428_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_12428_gb300 import build
    build.build()
    import paper_2502_12428_gb300.qfs as q
    return q


@pytest.mark.parametrize("p,n", [(5, 6000), (7, 1500), (11, 8)])
def test_noalloc_matches_heights_on_two_calls_in_a_row(qfs, p, n):
    a = torch.from_numpy(inputs.dense(p, n, 8800 + p)).cuda()
    b = torch.from_numpy(inputs.sparse(p, n, 8900 + p)).cuda()
    want_a = qfs.heights(p, a).cpu().numpy()
    want_b = qfs.heights(p, b).cpu().numpy()
    # two calls in a row on different batches: the second sees whatever the first left in the shared scratch
    got_a = qfs.heights_noalloc(p, a).cpu().numpy()
    got_b = qfs.heights_noalloc(p, b).cpu().numpy()
    assert np.array_equal(got_a, want_a)
    assert np.array_equal(got_b, want_b)
    assert (want_a != 1).any()


def test_noalloc_does_not_allocate(qfs):
    p = 5
    a = torch.from_numpy(inputs.dense(p, 3000, 8700)).cuda()
    out = torch.empty(3000, dtype=torch.int8, device="cuda")
    qfs.heights_noalloc(p, a, out=out)          # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        qfs.heights_noalloc(p, a, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(out.cpu().numpy(), qfs.heights(p, a).cpu().numpy())


def test_noalloc_rejects_sizes_beyond_the_array(qfs):
    a = torch.from_numpy(inputs.dense(13, 4, 1)).cuda()
    with pytest.raises(qfs.QfsError) as e:
        qfs.heights_noalloc(13, a)
    assert e.value.status == 5
    with pytest.raises(qfs.QfsError) as e:
        qfs.heights_noalloc(5, a, max_h=0)
    assert e.value.status == 2
