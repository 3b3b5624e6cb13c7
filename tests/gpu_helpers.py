"""Helpers for the GPU parity tests: moving seeded inputs to the device and
reading results back as Python integers for comparison with the oracle."""

import numpy as np
import torch

import paper_2402_00675_gb300 as mg

_SIGNED = (1, 3, 4)


def np_dtype(variant, width):
    if width == 32:
        return np.int32 if variant in _SIGNED else np.uint32
    return np.int64 if variant in _SIGNED else np.uint64


def dev(ints, dtype, pad_front=0):
    """Python ints -> CUDA tensor of `dtype`; with pad_front > 0 the returned
    view starts pad_front elements into a larger buffer (misaligned start)."""
    arr = np.array([int(x) for x in ints], dtype=np.int64 if dtype in (np.int32, np.int64) else np.uint64)
    arr = arr.astype(dtype)
    if pad_front:
        full = np.zeros(len(arr) + pad_front, dtype=dtype)
        full[pad_front:] = arr
        t = torch.from_numpy(full).cuda()
        return t[pad_front:]
    return torch.from_numpy(arr).cuda()


def dev_wide(ints, width, pad_front=0):
    """Double-width T values as device memory: int64/uint64 at width 32,
    two little-endian 64-bit words per value at width 64."""
    if width == 32:
        signed = any(x < 0 for x in ints)
        return dev(ints, np.int64 if signed else np.uint64, pad_front)
    words = []
    for x in ints:
        words.append(x & 0xFFFFFFFFFFFFFFFF)
        words.append((x >> 64) & 0xFFFFFFFFFFFFFFFF)
    return dev(words, np.uint64, 2 * pad_front)


def host(t):
    return [int(x) for x in t.cpu().numpy().tolist()]


def empty_like_elems(n, dtype, pad_front=0):
    torch_dtype = {np.int32: torch.int32, np.uint32: torch.uint32, np.int64: torch.int64,
                   np.uint64: torch.uint64}[dtype]
    t = torch.zeros(n + pad_front, dtype=torch_dtype, device="cuda")
    return t[pad_front:]


def sync():
    torch.cuda.synchronize()


def log2R_of(variant, width):
    return 2 * width if variant in (2, 3, 4) else width


def input_range(variant, N):
    """Inclusive range of mont_mul inputs (the variant's output range)."""
    if variant in (0, 2):
        return 0, N - 1
    if variant == 1:
        return -(N - 1), N - 1
    return -((N - 1) // 2), (N - 1) // 2


def max_modulus(variant, width, alpha=1):
    """Largest odd N the variant admits at this width."""
    import oracle as o
    l = log2R_of(variant, width)
    if variant == 0:
        N = (1 << width) - 1
    elif variant == 1:
        N = (1 << (width - 1)) - 1
    elif variant == 2:
        N = int((1 << width) / 1.6180339887498949) | 1
        while not o.plantard_bound_ok(N, width):
            N -= 2
        while o.plantard_bound_ok(N + 2, width):
            N += 2
    elif variant == 3:
        N = (1 << (width - 1)) - 1
    else:
        N = (1 << (width - alpha - 1)) - 1
    assert o.precondition_ok(variant, N, l, alpha)
    return N
