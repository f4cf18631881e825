"""Test helpers: tensor <-> numpy views with the ABI's key types."""
import numpy as np
import torch

NP_KEY = {"u32": np.uint32, "i32": np.int32, "u64": np.uint64, "f32": np.float32}


def to_np(t: torch.Tensor, kt: str | None = None) -> np.ndarray:
    """Host numpy copy; int32 tensors viewed as uint32 for u32 keys and payloads."""
    a = t.detach().cpu().numpy()
    if kt is not None:
        return a.view(NP_KEY[kt]) if a.dtype.itemsize == np.dtype(NP_KEY[kt]).itemsize else a.astype(NP_KEY[kt])
    return a


def vals_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def first_mismatch(x: np.ndarray, y: np.ndarray):
    bad = np.nonzero(x != y)[0]
    return None if len(bad) == 0 else int(bad[0])


def stable_merge_violation(A, B, C, Cv, unsigned=False, chunk=1 << 24):
    """First place where C / Cv fail to be the stable merge of A and B, or
    None.  Payloads must be the tags (src << 31) | index of the inputs (as
    the workloads make them).  Works on torch tensors of any device, in
    chunks, so it checks outputs of any size without a reference output:

    * every output's tag names an input element (index below its side's
      length) and the output's key is that element's key;
    * along C the pair (key, tag) strictly increases: keys non-decreasing,
      and on equal keys every A element (tag bit 31 clear) before every B
      element, each side in index order (the stability of Section 2).

    n + m distinct input elements in that order are exactly the unique
    stable merge.  `unsigned` compares 32-bit keys stored in int32 tensors
    as unsigned.  Returns (position, reason)."""
    import torch
    n, m, total = A.numel(), B.numel(), C.numel()
    if total != n + m or Cv.numel() != total:
        return (0, "length")
    prev_key = prev_tag = None
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        key = C[s:e]
        tag = Cv[s:e].to(torch.int64) & 0xFFFFFFFF
        from_b = (tag >> 31).bool()
        idx = tag & 0x7FFFFFFF
        bad = torch.nonzero(idx >= torch.where(from_b, m, n))
        if bad.numel():
            return (s + int(bad[0]), "tag names no input element")
        src_key = torch.empty_like(key)
        src_key[~from_b] = A[idx[~from_b]]
        src_key[from_b] = B[idx[from_b]]
        bad = torch.nonzero(src_key != key)
        if bad.numel():
            return (s + int(bad[0]), "key differs from its tagged input element")
        if unsigned:
            key = key.to(torch.int64) & 0xFFFFFFFF
        if prev_key is not None:
            key = torch.cat([prev_key, key])
            tag = torch.cat([prev_tag, tag])
        lo_k, hi_k, lo_t, hi_t = key[:-1], key[1:], tag[:-1], tag[1:]
        bad = torch.nonzero(~((lo_k < hi_k) | ((lo_k == hi_k) & (lo_t < hi_t))))
        if bad.numel():
            return (s + int(bad[0]) - (1 if prev_key is not None else 0), "order of (key, tag)")
        prev_key, prev_tag = key[-1:], tag[-1:]
    return None


def stable_sort_violation(src_keys, keys, vals, unsigned=False, chunk=1 << 24):
    """First place where (keys, vals) fail to be the stable sort of
    src_keys with payload = original index, or None.  Torch tensors of any
    device, checked in chunks: every payload is an index of src_keys whose
    key the output carries, and (key, index) strictly increases along the
    output (keys non-decreasing, equal keys in input order).  n distinct
    indices in that order are exactly the unique stable sort.  Returns
    (position, reason)."""
    import torch
    n = src_keys.numel()
    if keys.numel() != n or vals.numel() != n:
        return (0, "length")
    prev_key = prev_idx = None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        key = keys[s:e]
        idx = vals[s:e].to(torch.int64) & 0xFFFFFFFF
        bad = torch.nonzero(idx >= n)
        if bad.numel():
            return (s + int(bad[0]), "payload is no input index")
        bad = torch.nonzero(src_keys[idx] != key)
        if bad.numel():
            return (s + int(bad[0]), "key differs from the input element its payload names")
        if unsigned:
            key = key.to(torch.int64) & 0xFFFFFFFF
        if prev_key is not None:
            key = torch.cat([prev_key, key])
            idx = torch.cat([prev_idx, idx])
        lo_k, hi_k, lo_i, hi_i = key[:-1], key[1:], idx[:-1], idx[1:]
        bad = torch.nonzero(~((lo_k < hi_k) | ((lo_k == hi_k) & (lo_i < hi_i))))
        if bad.numel():
            return (s + int(bad[0]) - (1 if prev_key is not None else 0), "order of (key, index)")
        prev_key, prev_idx = key[-1:], idx[-1:]
    return None
