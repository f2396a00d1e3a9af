"""Helpers for the GPU parity tests (moving numpy arrays to and from CUDA)."""
import numpy as np
import torch


def cuda(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def same(a, b) -> bool:
    a = host(a) if isinstance(a, torch.Tensor) else np.asarray(a)
    b = host(b) if isinstance(b, torch.Tensor) else np.asarray(b)
    return a.shape == b.shape and np.array_equal(a, b)


def sorted_kpa_on_device(key_col: torch.Tensor, base: int, keys: torch.Tensor, ptrs: torch.Tensor):
    """The sorted-KPA invariants evaluated with torch ops on the device, for
    sizes the oracle cannot sort: (key, ptr) order, every row once, and
    key[i] = key_col[ptr[i]]."""
    n = keys.numel()
    assert ptrs.numel() == n
    if n == 0:
        return
    sk = (keys.view(torch.int64) ^ torch.iinfo(torch.int64).min)  # order-preserving signed view
    rel = ptrs.to(torch.int64) - base
    assert int(rel.min()) >= 0 and int(rel.max()) < n, "ptr out of range"
    seen = torch.zeros(n, dtype=torch.int32, device=keys.device)
    seen.index_fill_(0, rel, 1)
    assert int(seen.sum()) == n, "not a permutation"
    assert torch.equal(key_col.view(torch.int64)[rel], keys.view(torch.int64)), "key does not match its row"
    lt = sk[1:] > sk[:-1]
    eq = sk[1:] == sk[:-1]
    assert bool((lt | eq).all()), "keys not ascending"
    assert bool((~eq | (rel[1:] > rel[:-1])).all()), "equal keys not in ptr order"
