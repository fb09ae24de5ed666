"""Measured parity errors: printed, and appended as JSON lines to $SBHA_PARITY_LOG when it is set."""
import json
import os


def report(test: str, **values) -> None:
    line = {"test": test, **{k: (float(v) if hasattr(v, "__float__") and not isinstance(v, (bool, int, str)) else v)
                             for k, v in values.items()}}
    print("PARITY", json.dumps(line))
    path = os.environ.get("SBHA_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")


def col_rel_err(P, P_ref, mask=None):
    """max over columns j of max_i |P_ij - P_ref_ij| / max_i |P_ref_ij| (entries in mask only)."""
    import numpy as np

    d = np.abs(P - P_ref)
    if mask is not None:
        d = d * mask
    scale = np.abs(P_ref).max(axis=0)
    scale[scale == 0] = 1.0
    return float((d.max(axis=0) / scale).max())


def gram_rel_err(Z, Z_ref):
    """max |Z Z^T - Z_ref Z_ref^T| / max |Z_ref Z_ref^T| (unique where eigen-directions are not)."""
    import numpy as np

    G1, G2 = Z @ Z.T, Z_ref @ Z_ref.T
    return float(np.abs(G1 - G2).max() / np.abs(G2).max())
