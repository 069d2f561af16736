"""C-ABI checks that need no GPU: the library builds and loads, exports every entry
point include/bks.h declares, rejects bad arguments before touching the device, and
its host start-block generator agrees bit for bit with the oracle's own
implementation of the same published generator."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import rng as orng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    with open(os.path.join(ROOT, "include", "bks.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bks_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_05477_gb300 import _binding
    return _binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1504_05477_gb300 import _binding
    assert sorted(_binding.SIGNATURES) == _header_functions()


def test_version_and_strings(lib):
    assert lib.bks_version() >= 100
    assert lib.bks_status_string(0) == b"ok"
    assert lib.bks_status_string(1) == b"invalid argument"


def test_host_generator_matches_oracle_bitwise():
    from paper_1504_05477_gb300 import gen_pi_host
    for seed, d, k in [(0, 7, 3), (12345, 400, 10), (2**63 + 5, 33, 5)]:
        a = gen_pi_host(seed, d, k)
        b = orng.start_block(seed, d, k)
        assert a.dtype == np.float32 and a.shape == (d, k)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_invalid_arguments_rejected_without_device(lib):
    from paper_1504_05477_gb300 import _binding as B
    m = B.BksMatrix()
    m.kind = B.BKS_DENSE
    m.dtype = B.BKS_F32
    m.n, m.d, m.ld = 10, 5, 5
    m.vals = 1024   # never dereferenced: validation fails first
    null = ctypes.c_void_p()
    # no context
    assert lib.bks_block_krylov(null, ctypes.byref(m), 2, 1, 0, None, None, None, None, None,
                                None) == B.BKS_ERR_INVALID_ARG
    # bad sizes through the workspace query (pure host arithmetic)
    sz = ctypes.c_size_t()
    assert lib.bks_workspace_size(ctypes.byref(m), 0, 1, 0, None, ctypes.byref(sz)) == B.BKS_ERR_INVALID_ARG
    assert lib.bks_workspace_size(ctypes.byref(m), 6, 1, 0, None, ctypes.byref(sz)) == B.BKS_ERR_INVALID_ARG
    assert lib.bks_workspace_size(ctypes.byref(m), 2, -1, 0, None, ctypes.byref(sz)) == B.BKS_ERR_INVALID_ARG
    assert lib.bks_workspace_size(ctypes.byref(m), 2, 3, 0, None, ctypes.byref(sz)) == B.BKS_OK
    assert sz.value > 0
    assert lib.bks_gen_pi_host(0, 0, 3, None) == B.BKS_ERR_INVALID_ARG


def test_workspace_grows_with_width(lib):
    from paper_1504_05477_gb300 import _binding as B
    m = B.BksMatrix()
    m.kind, m.dtype = B.BKS_DENSE, B.BKS_F32
    m.n, m.d, m.ld = 20000, 8000, 8000
    sizes = []
    for q in (0, 4, 8):
        sz = ctypes.c_size_t()
        assert lib.bks_workspace_size(ctypes.byref(m), 50, q, 0, None, ctypes.byref(sz)) == 0
        sizes.append(sz.value)
    assert sizes[0] < sizes[1] < sizes[2]
    # Q (w x n) and B (w x d) at w = 450 are inside the plan
    assert sizes[2] > 450 * (20000 + 8000) * 4


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = ctypes.c_void_p()
    assert lib.bks_create(ctypes.byref(p), 0) != 0
