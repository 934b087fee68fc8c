"""The allocation-free key sort (sfg_sort_keys_static) against sfg_build.

Some callers cannot allocate device memory when they call into the library:
their device memory is reserved up front by their own pool, or they run a
latency-bound loop where cudaMalloc could block the host.  For them the
library offers a variant of the first build stage -- frame, Morton keys and
their stable sort -- whose temporaries live in one fixed device array.  This
test calls it through the C ABI twice in a row (the shared array keeps the
previous call's contents) and checks both results bit for bit against the
keys and order that sfg_build exports for the same particles.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

SFG_STATIC_MAX_N = 1 << 19


def _lib():
    import paper_2010_11254_gb300 as sfg
    lib = sfg._load()
    f = lib.sfg_sort_keys_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return sfg, f


def test_static_key_sort_matches_build_on_two_calls():
    import torch
    sfg, sort_static = _lib()
    clouds = [gen.uniform_cloud(70001, seed=21, n_sink=3),
              gen.clumpy_cloud(40000, n_clumps=32, n_sink=8, seed=22)]
    for c in clouds:
        pos = torch.from_numpy(c.pos).cuda()
        keys = torch.empty(c.n, dtype=torch.int64, device="cuda")
        order = torch.empty(c.n, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = sort_static(pos.data_ptr(), c.n, keys.data_ptr(), order.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == sfg.SFG_OK
        tree = sfg.Tree(pos, torch.from_numpy(c.mass).cuda(), torch.from_numpy(c.soft).cuda(),
                        torch.from_numpy(c.is_sink).cuda())
        np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), tree.export(sfg.FIELD_KEYS))
        np.testing.assert_array_equal(order.cpu().numpy(), tree.export(sfg.FIELD_ORDER))
        tree.close()


def test_static_key_sort_at_the_array_capacity():
    """n = SFG_STATIC_MAX_N fills every region of the fixed array exactly."""
    import torch
    sfg, sort_static = _lib()
    c = gen.uniform_cloud(SFG_STATIC_MAX_N, seed=23, n_sink=0)
    pos = torch.from_numpy(c.pos).cuda()
    tree = sfg.Tree(pos, torch.from_numpy(c.mass).cuda(), torch.from_numpy(c.soft).cuda())
    want_k, want_o = tree.export(sfg.FIELD_KEYS), tree.export(sfg.FIELD_ORDER)
    tree.close()
    for _ in range(2):
        keys = torch.empty(c.n, dtype=torch.int64, device="cuda")
        order = torch.empty(c.n, dtype=torch.int32, device="cuda")
        rc = sort_static(pos.data_ptr(), c.n, keys.data_ptr(), order.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == sfg.SFG_OK
        np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), want_k)
        np.testing.assert_array_equal(order.cpu().numpy(), want_o)


def test_static_key_sort_rejects_sizes_beyond_its_array():
    import torch
    sfg, sort_static = _lib()
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    rc = sort_static(pos.data_ptr(), SFG_STATIC_MAX_N + 1, out.data_ptr(), out.data_ptr(), None)
    assert rc == sfg.SFG_EINVAL
    rc = sort_static(pos.data_ptr(), 0, out.data_ptr(), out.data_ptr(), None)
    assert rc == sfg.SFG_EINVAL
