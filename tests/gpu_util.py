"""Helpers for the -m gpu tests: run the CUDA path through the C ABI on numpy inputs."""

import numpy as np

NORM_TO_ORACLE = {"per_level": "per_level", "end": "end", "none": "none"}


def run_forward(chw, torch, x, m, dtype="f32", norm="end", flags=0, adjoint=False, diag=None, inplace=False):
    """Transform the rows of numpy array x (batch, 2^m) on cuda:0; returns numpy."""
    dev = torch.device("cuda:0")
    batch = x.shape[0]
    p = chw.chw_plan(m, batch, dtype, norm, flags)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    yd = xd if inplace else torch.empty_like(xd)
    dd = None if diag is None else torch.from_numpy(diag).to(dev)
    if adjoint:
        chw.chw_adjoint(p, xd, yd, diag=dd)
    else:
        chw.chw_forward(p, xd, yd, diag=dd)
    torch.cuda.synchronize()
    st = chw.chw_last_device_status(p)
    assert st == 0, chw.chw_status_string(st)
    out = yd.cpu().numpy()
    info = chw.chw_plan_get_info(p)
    p.close()
    return out, info


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype.itemsize == 4 else a.view(np.uint16)


def assert_bitwise(got, ref, what=""):
    g, r = bits(got), bits(ref)
    if not np.array_equal(g, r):
        bad = np.argwhere(g != r)
        i = tuple(bad[0])
        raise AssertionError(
            f"{what}: {len(bad)} elements differ; first at {i}: got {got[i]!r} ref {ref[i]!r}"
        )
