"""The allocation-free connectivity call (snnmap_connectivity_noalloc) gives
the oracle's Conn (Eq. connectivity), as the handle-based
snnmap_connectivity does.

Some callers cannot allocate device memory at all: their device memory is
reserved up front by another allocator, or they run in a loop where a
cudaMalloc/cudaFree (which can synchronize the device) is not allowed. This
entry point serves them from a fixed static device array. The test calls it
through the C ABI twice in a row on the same inputs and on new ones, so a
second call must not see the first call's leftovers, and checks that inputs
beyond the array's capacity are refused before any work is queued. This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import snngen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2609_07577_gb300 as P
    return P


def _noalloc(P, hg, off, pins, w, rho, K, out):
    L = P.lib()
    rc = L.snnmap_connectivity_noalloc(hg.V, hg.E, off.data_ptr(), pins.data_ptr(), w.data_ptr(),
                                       rho.data_ptr(), K, out.data_ptr(), None)
    assert rc == 0, L.snnmap_last_error()
    torch.cuda.synchronize()
    return int(out.item())


def test_noalloc_matches_connectivity(lib):
    P = lib
    rng = np.random.default_rng(11)
    for name in ("cfg1", "cfg3s"):
        hg = snngen.by_name(name)
        off = torch.from_numpy(hg.off).cuda()
        pins = torch.from_numpy(hg.pins).cuda()
        w = torch.from_numpy(hg.w).cuda()
        g = P.HGraph(P.params_for(hg.omega, hg.delta, hg.phi), hg.V, off, pins, w)
        out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        try:
            for K in (97, 97, 5, hg.V):
                rho = torch.from_numpy(rng.integers(0, K, size=hg.V).astype(np.int32)).cuda()
                ref = P.snnmap_connectivity(g.handle, K, rho)
                # Eq. connectivity from the oracle on the same partition
                orc = oracle.Level.from_hypergraph(hg, oracle.params_of(hg)).conn(rho.cpu().numpy())
                first = _noalloc(P, hg, off, pins, w, rho, K, out)
                second = _noalloc(P, hg, off, pins, w, rho, K, out)
                assert ref == orc, (name, K, ref, orc)
                assert first == orc and second == orc, (name, K, first, second, orc)
        finally:
            g.close()


def test_noalloc_refuses_oversized_input(lib):
    P = lib
    hg = snngen.by_name("cfg1s")
    off = torch.from_numpy(hg.off).cuda()
    pins = torch.from_numpy(hg.pins).cuda()
    w = torch.from_numpy(hg.w).cuda()
    rho = torch.zeros(hg.V, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    L = P.lib()
    rc = L.snnmap_connectivity_noalloc(hg.V, (1 << 22) + 1, off.data_ptr(), pins.data_ptr(),
                                       w.data_ptr(), rho.data_ptr(), 1, out.data_ptr(), None)
    assert rc == 1
    assert b"4194304" in L.snnmap_last_error()
