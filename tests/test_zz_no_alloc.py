"""cmc_potential_static, the allocation-free variant of cmc_potential.

Callers that may not allocate device memory (allocation-free real-time
loops, programs that own all device memory through their own pool, plug-ins
whose host application owns the allocator) use this entry point; its scratch
is a fixed array of the library's device memory.  It must give what cmc_potential
gives, call after call, even though every call reuses the same array.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, host, sorted_plummer

pytestmark = pytest.mark.gpu


def test_static_potential_equals_allocating_potential_on_consecutive_calls(orc):
    import torch

    import paper_1206_5878_gb300 as g
    lib = g.load()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row; the second is smaller, so stale tile sums left by
    # the first call would show up if the scratch were read before written
    for n, seed, masses in ((100_003, 1, "salpeter"), (4_097, 2, "equal")):
        s = sorted_plummer(n, seed=seed, masses=masses)
        r, m = dev(s["r"]), dev(s["m"])
        phi_ref, M_ref = g.stage_potential(r, m, want_M=True)
        phi = torch.full_like(r, np.nan)
        M = torch.full_like(r, np.nan)
        st = lib.cmc_potential_static(n, r.data_ptr(), m.data_ptr(), phi.data_ptr(),
                                      M.data_ptr(), stream)
        assert st == 0
        torch.cuda.synchronize()
        a, b = host(phi), host(phi_ref)
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a / b - 1)) < 1e-12  # the potential tests' tolerance
        assert np.max(np.abs(host(M) / host(M_ref) - 1)) < 1e-12
        # and the oracle agrees
        assert np.max(np.abs(a / orc.potential(s["r"], s["m"], "dd") - 1)) < 1e-12
    # a call after the first on this device takes no device memory: the
    # free memory the driver reports is the same before and after it
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert lib.cmc_potential_static(n, r.data_ptr(), m.data_ptr(), phi.data_ptr(),
                                    M.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_array_equal(host(phi), a)  # and repeats its bits


def test_static_potential_limits():
    import torch

    import paper_1206_5878_gb300 as g
    lib = g.load()
    r = torch.ones(8, dtype=torch.float64, device="cuda")
    # too many stars for the fixed scratch: rejected before any launch
    assert lib.cmc_potential_static((1 << 24) + 1, r.data_ptr(), r.data_ptr(), r.data_ptr(),
                                    None, None) == 1
    assert lib.cmc_potential_static(0, None, None, None, None, None) == 0
    assert lib.cmc_potential_static(-1, None, None, None, None, None) == 1
