"""The allocation-free sampled count against the regular one and the oracle
(needs a GPU).

mochy_count_sampled_noalloc serves callers that cannot allocate device memory
while they run; it keeps its working memory in one fixed array inside the
library, shared by all calls.  Two calls in a row (different methods, sample
counts and seeds) must each give, bit for bit, what mochy_count_sampled and
the oracle give on the same Philox draws: raw counts equal as int64 and FP64
estimates equal (both sides scale the same integers by the same operations
in the same order).  This file is collected last and also runs alone in a
fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import binding as B, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    spec = synth.HypergraphSpec(500, 1000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)
    off, nodes = synth.generate(spec)
    with B.Context() as ctx:
        ctx.load(spec.n_nodes, off, nodes)
        ctx.project()
        stream = torch.cuda.ExternalStream(ctx.stream)
        for method, samples, seed in ((B.MOCHY_A_PLUS, 3000, 17), (B.MOCHY_A, 300, 2**33 + 1)):
            raw_h = torch.full((26,), -1, dtype=torch.int64, device="cuda")
            raw_3h = torch.full((431,), -1, dtype=torch.int64, device="cuda")
            est_h = torch.full((26,), -1.0, dtype=torch.float64, device="cuda")
            est_3h = torch.full((431,), -1.0, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            before = B.mochy_device_bytes(ctx.h)
            B.mochy_count_sampled_noalloc(ctx.h, method, samples, seed, raw_h.data_ptr(),
                                          raw_3h.data_ptr(), est_h.data_ptr(), est_3h.data_ptr())
            stream.synchronize()
            assert B.mochy_device_bytes(ctx.h) == before        # nothing allocated
            got = (raw_h.cpu().numpy(), raw_3h.cpu().numpy(), est_h.cpu().numpy(),
                   est_3h.cpu().numpy())
            ref = ctx.count_sampled(method, samples, seed)
            orc = oracle.count_sampled(off, nodes, method, samples, seed)
            for a, b, o in zip(got, ref, orc):
                assert np.array_equal(a, b)
                assert np.array_equal(a, o)
            assert ref[0].sum() > 0


def test_noalloc_rejects_too_many_samples():
    import torch
    off, nodes = synth.generate(synth.TINY)
    with B.Context() as ctx:
        ctx.load(synth.TINY.n_nodes, off, nodes)
        ctx.project()
        out = [torch.zeros(n, dtype=t, device="cuda") for n, t in
               ((26, torch.int64), (431, torch.int64), (26, torch.float64), (431, torch.float64))]
        with pytest.raises(B.MochyError) as e:
            B.mochy_count_sampled_noalloc(ctx.h, B.MOCHY_A, 65537, 1, *[o.data_ptr() for o in out])
        assert e.value.code == B.E_UNSUPPORTED
