"""Helpers shared by the GPU parity tests (tensor transfer, error norms and
the measured figures reported at the end of the run)."""
import numpy as np
import torch

# Figures the tests measured (errors, ratios against the oracle), listed by
# the terminal summary of the run (tests/conftest.py), so that they appear in
# the output of a quiet run.
NOTES = []


def note(*parts):
    text = " ".join(str(p) for p in parts)
    NOTES.append(text)
    print(text)


def dev(x, dtype=None):
    x = np.asarray(x)
    if dtype is None:
        dtype = torch.complex64 if np.iscomplexobj(x) else (torch.int32 if x.dtype.kind in "iu" else torch.float32)
    return torch.as_tensor(x).to(dtype).cuda().contiguous()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def rel_l2(got, ref, mask=None):
    got = np.asarray(got)
    ref = np.asarray(ref)
    if mask is not None:
        got, ref = got[mask], ref[mask]
    den = np.sqrt(np.sum(np.abs(ref) ** 2))
    return float(np.sqrt(np.sum(np.abs(got - ref) ** 2)) / max(den, 1e-300))
