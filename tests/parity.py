"""Block-by-block comparison of a GPU reconstruction with the oracle's.

The oracle reports, for every block, its selection sequence and the FP64
relative gap between the chosen score and the best other one.  A GPU block
matches when its selection sequence equals the oracle's, or the oracle's
conjugate mirror k -> -k mod W (with real data, R(-k) = conj R(k), so the
mirror trajectory gives the same real output), and its 16 output pixels are
within ``tol`` (max-abs).  A block whose sequence departs from the oracle's is
accepted only if the oracle's own record shows a near-tie (gap < ``tie``) at
the first iteration where they differ; such blocks are counted and returned.
"""
import numpy as np

W = 32


def mirror(k):
    k = np.asarray(k)
    return ((-(k // W)) % W) * W + ((-(k % W)) % W)


def _prefix(a, b):
    neq = np.nonzero(a != b)[0]
    return len(a) if len(neq) == 0 else int(neq[0])


def compare(gpu_hr, gpu_sel, orc_hr, orc_sel, orc_gap, blocks, nbw, tol=1e-4, tie=1e-4,
            gpu_dc=None, orc_dc=None, dc_tol=1e-3):
    """Returns dict(n, matched, near_ties, max_err, fails, tie_blocks)."""
    gpu_sel = np.asarray(gpu_sel).astype(np.int64) & 0xFFFF
    out = dict(n=len(blocks), matched=0, near_ties=0, max_err=0.0, fails=[], tie_blocks=[])
    for i, b in enumerate(blocks):
        bi, bj = divmod(int(b), nbw)
        g = gpu_hr[4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
        o = orc_hr[4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
        err = float(np.max(np.abs(g.astype(np.float64) - o)))
        sg, so = gpu_sel[i], np.asarray(orc_sel[i])
        ld, lm = _prefix(sg, so), _prefix(sg, mirror(so))
        L = max(ld, lm)
        if L == len(so):
            dc_ok = True
            if gpu_dc is not None:
                ref = orc_dc[i] if ld >= lm else np.conj(orc_dc[i])
                dc_ok = float(np.max(np.abs(gpu_dc[i] - ref))) <= dc_tol
            if err <= tol and dc_ok:
                out["matched"] += 1
                out["max_err"] = max(out["max_err"], err)
            else:
                out["fails"].append((int(b), "same sequence, err %.3g, dc_ok %s" % (err, dc_ok)))
        elif orc_gap[i][L] < tie:
            out["near_ties"] += 1
            out["tie_blocks"].append((int(b), L, float(orc_gap[i][L]), err))
        else:
            out["fails"].append((int(b), "sequence differs at %d, oracle gap %.3g, err %.3g"
                                 % (L, orc_gap[i][L], err)))
    return out
