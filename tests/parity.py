"""The gradient comparison of the GPU <-> oracle parity protocol.

A group passes when ||g_gpu - g_oracle|| <= rtol ||g_oracle|| and, element by
element on the entries with |g_oracle| >= 1e-2 max |g_oracle| of the group,
|g_gpu - g_oracle| <= rtol |g_oracle| (so that a few wrong entries cannot
hide inside a large group).  A group whose oracle gradient is exactly zero
must be (nearly) zero on the GPU too."""
import numpy as np


def group_errors(a, b):
    """(norm-relative error, largest per-element relative error on the
    entries >= 1e-2 of the group's largest, number of such entries)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a)), 0.0, 0
    big = np.abs(b) >= 1e-2 * np.abs(b).max()
    el = np.abs(a - b)[big] / np.abs(b)[big]
    return float(np.linalg.norm(a - b) / nb), float(el.max()), int(big.sum())


def compare_grads(gg, go, groups, rtol=1e-3):
    for k in groups:
        a = gg[k].cpu().numpy() if hasattr(gg[k], "cpu") else gg[k]
        b = np.asarray(go[k], np.float64)
        if np.linalg.norm(b) == 0.0:
            assert np.linalg.norm(np.asarray(a, np.float64)) <= 1e-6, k
            continue
        norm_err, el_err, n_big = group_errors(a, b)
        assert norm_err <= rtol, (k, "group", norm_err)
        assert el_err <= rtol, (k, "element", el_err, n_big)
