"""The allocation-free variant of the bit-vector column kernel.

Some callers cannot allocate device memory: a process whose device memory is all reserved by
another allocator's pool (a cudaMalloc there fails or takes memory the pool counts on), or a
latency-critical path that must not pay an allocation's implicit synchronization.  For them
peanut_bitvector_columns_noalloc takes only caller-owned device buffers and keeps its scratch in
a fixed array inside the library.  This file checks, through the C ABI, that it returns exactly
what the allocating entry point (peanut_debug_bitvector_columns) returns, and that both equal the
oracle's DP column, on two calls in a row, and that a request larger than the fixed scratch is
refused.  It is collected last on purpose.
"""
import ctypes
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _cases(seed):
    rng = random.Random(seed)
    pats, txts = [], []
    for m in (1, 2, 17, 63, 64, 65, 100, 127, 128, 129, 191, 192, 193, 250, 255):
        for _ in range(3):
            p = "".join(rng.choice("ACGT") for _ in range(m))
            src = list(p)
            for _ in range(rng.randint(0, 3)):
                src[rng.randrange(len(src))] = rng.choice("ACGT")
            t = ("".join(rng.choice("ACGT") for _ in range(rng.randint(0, 30))) + "".join(src)
                 + "".join(rng.choice("AC") for _ in range(rng.randint(1, 30))))
            pats.append(p.encode())
            txts.append(t.encode())
    return pats, txts


def _device_buffers(pats, txts):
    import torch
    po = np.zeros(len(pats) + 1, np.int64)
    po[1:] = np.cumsum([len(p) for p in pats])
    to = np.zeros(len(txts) + 1, np.int64)
    to[1:] = np.cumsum([len(t) for t in txts])
    d = lambda a: torch.from_numpy(a).cuda()
    return (d(np.frombuffer(b"".join(pats), np.uint8).copy()), d(po),
            d(np.frombuffer(b"".join(txts), np.uint8).copy()), d(to),
            torch.full((int(to[-1]),), -1, dtype=torch.int32, device="cuda"), to)


def test_noalloc_equals_allocating_entry_point_twice(gpu):
    import oracle
    import torch
    lib = gpu.load()
    for seed in (11, 12):  # two calls in a row, different inputs
        pats, txts = _cases(seed)
        want = gpu.bitvector_columns(pats, txts)
        # the allocating entry point itself equals the oracle's DP column (Section "Validation")
        for p, t, w in zip(pats, txts, want):
            assert w.tolist() == oracle.semiglobal_column(p, t).tolist()
        dp, dpo, dt, dto, dout, to = _device_buffers(pats, txts)
        st = lib.peanut_bitvector_columns_noalloc(dp.data_ptr(), dpo.data_ptr(), len(pats), dt.data_ptr(),
                                                  dto.data_ptr(), dout.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream)
        assert st == 0, lib.peanut_last_error()
        got = dout.cpu().numpy()
        for i, w in enumerate(want):
            assert got[int(to[i]):int(to[i + 1])].tolist() == w.tolist(), (seed, i)


def test_noalloc_refuses_more_patterns_than_its_scratch(gpu):
    import torch
    lib = gpu.load()
    pats = [b"ACGT"] * 8193
    dp, dpo, dt, dto, dout, _ = _device_buffers(pats, pats)
    st = lib.peanut_bitvector_columns_noalloc(dp.data_ptr(), dpo.data_ptr(), len(pats), dt.data_ptr(),
                                              dto.data_ptr(), dout.data_ptr(), None)
    assert st == 1
    assert b"8192" in lib.peanut_last_error()
