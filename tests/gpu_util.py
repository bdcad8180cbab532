"""Helpers for the GPU tests: run hp pipelines on torch device memory."""

import numpy as np
import torch

from paper_2012_07145_gb300 import hp

TORCH_OF = {hp.HP_F32: torch.float32, hp.HP_F16: torch.float16, hp.HP_BF16: torch.bfloat16,
            hp.HP_U8: torch.uint8, hp.HP_U16: torch.int16, hp.HP_U32: torch.int32}  # u16 held as int16 bits


def to_device(arr: np.ndarray, dtype: int) -> torch.Tensor:
    """Upload a [C][H][W] numpy array (already in the right element type, or
    float values to round for f16/bf16)."""
    if dtype in (hp.HP_F16, hp.HP_BF16):
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).to(TORCH_OF[dtype])
    elif dtype == hp.HP_U16:
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint16).view(np.int16))
    else:
        t = torch.from_numpy(np.ascontiguousarray(arr))
    return hp.padded_copy(t)


def empty(c, h, w, dtype: int) -> torch.Tensor:
    return hp.padded_empty(c, h, w, TORCH_OF[dtype])


# Guard bands around an output: every row is followed by at least 16 bytes of
# padding, every plane by a whole padding row, and the image by GUARD bytes on
# each side; all of it holds CANARY before a realize and must hold it after.
GUARD = 256
CANARY = 0xA5


def guarded_empty(c: int, h: int, w: int, dtype: int, device="cuda") -> torch.Tensor:
    """A [C][H][W] output with the C ABI's 16-byte strides inside a canary-filled
    allocation (row padding, a guard row per plane, guard bytes before and after)."""
    tdt = TORCH_OF[dtype]
    es = torch.empty((), dtype=tdt).element_size()
    per = 16 // es
    wp = (w + per - 1) // per * per + per
    plane = wp * (h + 1)
    raw = torch.full((2 * GUARD + c * plane * es,), CANARY, dtype=torch.uint8, device=device)
    out = raw.view(tdt)[GUARD // es:].as_strided((c, h, w), (plane, wp, 1))
    out.guard = (raw, c, h, w * es, wp * es, plane * es)
    return out


def outside_writes(out: torch.Tensor) -> int:
    """Bytes outside the image of a guarded_empty output that no longer hold CANARY."""
    raw, c, h, wb, rs, ps = out.guard
    mask = torch.ones_like(raw, dtype=torch.bool)
    mask[GUARD:].as_strided((c, h, wb), (ps, rs, 1)).fill_(False)
    return int(((raw != CANARY) & mask).sum())


def run(p: hp.Pipeline, inputs, in_dtypes, out_shape, out_dtype, out=None) -> torch.Tensor:
    """Realize pipeline p on device tensors; returns the output tensor.  A new
    output is guarded: the realize must write nothing outside the image."""
    bufs = [hp.buffer_from_tensor(t, d) for t, d in zip(inputs, in_dtypes)]
    guarded = out is None
    if guarded:
        out = guarded_empty(*out_shape, out_dtype)
    # the inputs must come back unchanged (those that are not the output itself)
    kept = [(t, t.clone()) for t in inputs if t.data_ptr() != out.data_ptr()]
    p.realize(bufs, hp.buffer_from_tensor(out, out_dtype), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert p.device_error() == 0, "kernel reported a device-side error"
    if guarded:
        n = outside_writes(out)
        assert n == 0, f"the realize wrote {n} bytes outside its {tuple(out.shape)} output"
    for t, before in kept:
        assert torch.equal(bits(t), bits(before)), "the realize changed one of its inputs"
    return out


def to_numpy(t: torch.Tensor) -> np.ndarray:
    if t.dtype in (torch.float16, torch.bfloat16):
        return t.float().cpu().numpy()
    if t.dtype == torch.int16:
        return t.cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def bits(t: torch.Tensor) -> torch.Tensor:
    """Bit pattern of a float tensor, for bit-identity checks."""
    if t.dtype == torch.float32:
        return t.view(torch.int32)
    if t.dtype in (torch.float16, torch.bfloat16):
        return t.view(torch.int16)
    return t


def rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max |got - ref| / (max(ref) - min(ref)): the FP32 parity measure."""
    rng = float(ref.max() - ref.min())
    return float(np.abs(got.astype(np.float64) - ref).max() / (rng if rng > 0 else 1.0))


def u16_close(got: np.ndarray, ref_float: np.ndarray, delta_lsb: float = 0.25):
    """uint16 parity where float decides the integer: exact except where the
    oracle's value lies within delta_lsb of a rounding boundary, where one LSB
    either way is allowed.  Returns (ok, n_boundary_mismatches)."""
    scaled = np.clip(ref_float * 65535.0, 0, 65535)
    ref = np.clip(np.rint(scaled), 0, 65535).astype(np.int64)
    diff = np.abs(got.astype(np.int64) - ref)
    frac = np.abs(scaled - np.floor(scaled) - 0.5)
    near = frac < delta_lsb
    bad = (diff > 1) | ((diff == 1) & ~near)
    return (not bad.any()), int(((diff == 1) & near).sum())
