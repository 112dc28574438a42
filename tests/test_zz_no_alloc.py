"""nuri_hop_index_noalloc: the hop/label index built with no device memory allocated by the
call, for callers that cannot allocate at that point (GPU memory reserved up front by another
framework, a service thread that must not block or fail in an allocator, a recovery path after
an out-of-memory error).  Its output must equal that of the allocating path (nuri_load_graph
with index_hops, then nuri_hop_index), integer for integer, on two calls in a row: the second
call reuses the fixed scratch array the first one left behind.

This file is named to be collected last, so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import paper_1807_08888_b300 as nuri


def _graph(n, m, hubs, hub_deg, L, seed):
    """Random undirected graph with `hubs` vertices of degree about hub_deg (above the 2048
    entries that send a vertex to the block-per-vertex kernel), labels 0..L-1 (each present),
    weights 0..1000."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    hs, hd = [], []
    for h in range(hubs):
        nb = rng.choice(n, hub_deg, replace=False)
        hs.append(np.full(hub_deg, h))
        hd.append(nb)
    if hubs:
        src = np.concatenate([src] + hs)
        dst = np.concatenate([dst] + hd)
    labels = rng.integers(0, L, n).astype(np.uint8)
    labels[:L] = np.arange(L, dtype=np.uint8)  # every label present, so the label count is L
    weights = rng.integers(0, 1001, n).astype(np.int32)
    return src.astype(np.int32), dst.astype(np.int32), labels, weights


def _csr(n, src, dst):
    """Symmetric CSR without self-loops or duplicate entries (the adjacency load_graph
    builds), rows sorted."""
    keep = src != dst
    a = np.minimum(src[keep], dst[keep]).astype(np.int64)
    b = np.maximum(src[keep], dst[keep]).astype(np.int64)
    pairs = np.unique(a * n + b)
    a, b = pairs // n, pairs % n
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, rows + 1, 1)
    off = np.cumsum(off)
    return off, cols.astype(np.int32)


def _noalloc(torch, n, off, adj, labels, L, score, hops):
    dev = torch.device("cuda")
    t_off = torch.from_numpy(off).to(dev)
    t_adj = torch.from_numpy(adj).to(dev) if adj.size else torch.empty(1, dtype=torch.int32,
                                                                      device=dev)
    t_lab = torch.from_numpy(labels).to(dev)
    t_sc = torch.from_numpy(score).to(dev)
    out = torch.full((hops * n * L,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    rc = nuri.lib().nuri_hop_index_noalloc(
        int(n), ctypes.c_void_p(t_off.data_ptr()), ctypes.c_void_p(t_adj.data_ptr()),
        int(adj.size), ctypes.c_void_p(t_lab.data_ptr()), int(L),
        ctypes.c_void_p(t_sc.data_ptr()), int(hops), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == nuri.OK, nuri.lib().nuri_last_error()
    return out.cpu().numpy().reshape(hops, n, L)


@pytest.mark.gpu
def test_noalloc_hop_index_matches_allocating_path_twice():
    import torch
    cases = [
        # (n, random edges, hubs, hub degree, labels, hops, seed)
        (6000, 30000, 3, 3000, 8, 3, 11),   # hub rows take the block-per-vertex kernel
        (2500, 9000, 1, 2100, 3, 2, 12),    # fewer vertices: stale scratch from call 1 unused
    ]
    for n, m, hubs, hub_deg, L, hops, seed in cases:
        src, dst, labels, weights = _graph(n, m, hubs, hub_deg, L, seed)
        G = nuri.load_graph(n, src, dst, labels=labels, weights=weights, index_hops=hops)
        try:
            assert G.info()["num_labels"] == L
            ref = nuri.hop_index(G, hops)
        finally:
            G.free()
        off, adj = _csr(n, src, dst)
        got = _noalloc(torch, n, off, adj, labels, L, weights, hops)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.gpu
def test_noalloc_rejects_bad_input_without_writing():
    import torch
    n, L, hops = 100, 2, 2
    src, dst, labels, weights = _graph(n, 300, 0, 0, L, 5)
    off, adj = _csr(n, src, dst)
    bad = adj.copy()
    bad[7] = n + 3  # neighbour id out of range: found by the device check
    dev = torch.device("cuda")
    t = [torch.from_numpy(x).to(dev) for x in (off, bad, labels, weights)]
    out = torch.full((hops * n * L,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    rc = nuri.lib().nuri_hop_index_noalloc(
        n, ctypes.c_void_p(t[0].data_ptr()), ctypes.c_void_p(t[1].data_ptr()), int(bad.size),
        ctypes.c_void_p(t[2].data_ptr()), L, ctypes.c_void_p(t[3].data_ptr()), hops,
        ctypes.c_void_p(out.data_ptr()), None)
    assert rc == nuri.ERR_INVALID
    assert b"malformed CSR" in nuri.lib().nuri_last_error()
    assert bool((out == -7).all())


def test_noalloc_rejects_sizes_beyond_the_limit_before_any_cuda_call():
    L = nuri.lib()
    big = (1 << 20) + 1
    assert L.nuri_hop_index_noalloc(big, None, None, 0, None, 4, None, 2, None, None) == nuri.ERR_INVALID
    assert b"exceed the limit" in L.nuri_last_error()
    assert L.nuri_hop_index_noalloc(10, None, None, 0, None, 4, None, 9, None, None) == nuri.ERR_INVALID
    assert L.nuri_hop_index_noalloc(10, None, None, 0, None, 0, None, 2, None, None) == nuri.ERR_INVALID
