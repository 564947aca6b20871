"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np

# tolerances on max |dT| relative to max |T| (identical accepted sets required)
TOL = {"f64": 1e-12, "f32": 2e-5}

# oracle tags (Sec. 4.2) -> public tag classes of include/fmm.h
_ORACLE_TO_PUBLIC = np.array([0, 1, 1, 3, 2, 2], dtype=np.uint8)


def oracle_classes(G):
    return _ORACLE_TO_PUBLIC[G]


def compare(T_gpu, G_gpu, ref, dtype_name, width=np.inf, h=None):
    """Element-by-element comparison of a GPU solve with an oracle result.

    Tags must agree exactly (cells within the tolerance of width_band are
    excluded from the tag check, where either side may legitimately accept);
    values of accepted and FIX cells must agree within the dtype's tolerance
    relative to max |T|; FAR cells must be +inf on both sides."""
    T_ref, G_ref = ref["T"], oracle_classes(ref["G"])
    T_gpu = np.asarray(T_gpu, dtype=np.float64)
    G_gpu = np.asarray(G_gpu)
    fin = np.isfinite(T_ref)
    scale = float(np.max(np.abs(T_ref[fin]))) if fin.any() else 1.0
    tol = TOL[dtype_name] * max(scale, 1e-300)
    if np.isfinite(width):
        edge = np.abs(np.abs(T_ref) - width) <= tol * 4
    else:
        edge = np.zeros(T_ref.shape, bool)
    bad_tags = (G_gpu != G_ref) & ~edge
    assert not bad_tags.any(), (
        f"{int(bad_tags.sum())} tag mismatches, first at {np.argwhere(bad_tags)[:3].tolist()}: "
        f"gpu {G_gpu[bad_tags][:5]} oracle {G_ref[bad_tags][:5]}")
    acc = ((G_ref == 2) | (G_ref == 3)) & ~edge
    err = np.abs(T_gpu[acc] - T_ref[acc])
    worst = float(err.max()) if err.size else 0.0
    assert worst <= tol, f"max |dT| = {worst:.3e} > {tol:.3e} ({dtype_name}, max T {scale:.4g})"
    far = (G_ref == 0) & ~edge
    assert np.all(np.isinf(T_gpu[far]) & (T_gpu[far] > 0))
    # signs of accepted cells agree
    same_sign = (np.signbit(T_gpu[acc]) == np.signbit(T_ref[acc])) | (T_ref[acc] == 0)
    assert np.all(same_sign)
    return worst / max(scale, 1e-300)
