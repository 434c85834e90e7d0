"""Splits the export of a batch representation (smash_build_batch) into the
exports that each problem would have on its own, in the layout of
smash_export (node ids, sorted positions and caller indices local to the
problem).  Pure numpy; used by the batch parity tests."""
import numpy as np


def split_batch_export(e: dict, offsets) -> list:
    offsets = np.asarray(offsets, dtype=np.int64)
    T = len(offsets) - 1
    nn = len(e["level"])
    prob = np.asarray(e["node_problem"], dtype=np.int64)
    # local id of every node within its problem
    local = np.empty(nn, dtype=np.int64)
    for t in range(T):
        ids = np.nonzero(prob == t)[0]
        local[ids] = np.arange(len(ids))
    # per-node slices of the flat per-node arrays
    k_off = np.concatenate([[0], np.cumsum(e["k_row"])])
    mk = e["m_row"].astype(np.int64) - e["k_row"]
    r_off = np.concatenate([[0], np.cumsum(mk)])
    g_off = np.concatenate([[0], np.cumsum(mk * e["k_row"])])

    def remap(a):
        a = np.asarray(a, dtype=np.int64)
        return np.where(a < 0, a, local[np.maximum(a, 0)])

    out = []
    for t in range(T):
        o0, o1 = int(offsets[t]), int(offsets[t + 1])
        ids = np.nonzero(prob == t)[0]
        d = {}
        d["permx"] = e["permx"][o0:o1] - o0
        d["permy"] = d["permx"]
        d["keyx"] = e["keyx"][o0:o1]
        d["keyy"] = d["keyx"]
        lv = e["level"][ids]
        L = int(lv.max())
        d["lvl_off"] = np.concatenate([[0], np.cumsum([np.sum(lv == l) for l in range(1, L + 1)])]).astype(np.int64)
        d["L"] = L
        d["level"] = lv
        d["leaf"] = e["leaf"][ids]
        d["parent"] = remap(e["parent"][ids]).astype(np.int32)
        d["child0"] = remap(e["child0"][ids]).astype(np.int32)
        d["nchild"] = e["nchild"][ids]
        d["rs"] = e["rs"][ids] - o0
        d["cs"] = e["cs"][ids] - o0
        d["rc"] = e["rc"][ids]
        d["cc"] = e["cc"][ids]
        d["cell"] = e["cell"][ids]
        for name in ("adm", "near"):
            ptr, col = e[f"{name}_ptr"], e[f"{name}_col"]
            rows = [col[ptr[g]:ptr[g + 1]] for g in ids]
            d[f"{name}_ptr"] = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
            d[f"{name}_col"] = (np.concatenate(rows) if rows else np.zeros(0, np.int64))
            d[f"{name}_col"] = local[d[f"{name}_col"].astype(np.int64)].astype(np.int32)
        for tag in ("row", "col"):
            d[f"m_{tag}"] = e["m_row"][ids]
            d[f"k_{tag}"] = e["k_row"][ids]
            d[f"skel_{tag}"] = np.concatenate([e["skel_row"][k_off[g]:k_off[g + 1]] for g in ids]) - o0
            d[f"rest_{tag}"] = np.concatenate([e["rest_row"][r_off[g]:r_off[g + 1]] for g in ids]) - o0
            d[f"G_{tag}"] = np.concatenate([e["G_row"][g_off[g]:g_off[g + 1]] for g in ids])
        d["cube"] = e["problem_cube"][t]
        out.append(d)
    return out
