"""Write tests/golden/full_size.json: oracle logdet / chi2 / logL for sampled
columns of the full-size workloads (one N=1024 segment; the gap-free N=8192
batch of K=4096; the gapped three-detector N=16384 batch of K=1024; the
longest segment, N=32257, of the 64-segment mix; every pool column of the
serving workload's first gapped N=8192 and N=16384 segments).

Calls only the CPU oracle and the seeded input generators.  Run from the
repository root:  python tests/golden/make_golden.py [key ...]
(with keys, only those entries are recomputed and the others kept).
The N=32257 entry was written with OPENBLAS_NUM_THREADS=1: the threaded
OpenBLAS Cholesky of this host crashed at that size (about 4 min single-threaded).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_06010_b300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size.json")


def sample_cols(K, extra):
    cols = sorted(set([c for c in extra if c < K]))
    return cols


def one(n, fs, seed, K, rseed, cols, n_gaps=0, gap_len=512, scale=1.0):
    seg = inputs.make_segment(n, fs, seed, n_gaps=n_gaps, gap_len=gap_len, scale=scale)
    R = inputs.residual_batch(seg, K, rseed)
    osg = oracle.OracleSegment(seg.acf, seg.mask)
    sub = R[cols]
    chi = osg.chi2(sub)
    ll = oracle.loglike_from_chi2(chi, osg.logdet, osg.n_kept)
    return dict(n=n, fs=fs, seed=seed, K=K, rseed=rseed, n_gaps=n_gaps, gap_len=gap_len, scale=scale,
                n_kept=osg.n_kept, columns=cols, logdet=osg.logdet, chi2=chi.tolist(), logL=ll.tolist(),
                r_checksum=[float(np.sum(sub[i].astype(np.float64))) for i in range(len(cols))])


def mix64_longest():
    """Longest segment of the 64-segment mix, coloured-noise residuals of its own PSD."""
    specs = inputs.mix64_segments()
    i = max(range(len(specs)), key=lambda j: specs[j]["n"])
    sp = specs[i]
    rseed = sp["seed"] + 7
    acf = inputs.acf_from_psd(sp["n"], sp["fs"], a=sp["a"], floor=sp["floor"])
    R = inputs.noise_residuals(sp["n"], sp["fs"], sp["K"], rseed, a=sp["a"], floor=sp["floor"])
    cols = sample_cols(sp["K"], [0, 1, 2, 100, sp["K"] // 2, sp["K"] - 1])
    osg = oracle.OracleSegment(acf)
    sub = R[cols]
    chi = osg.chi2(sub)
    ll = oracle.loglike_from_chi2(chi, osg.logdet, osg.n_kept)
    return dict(index=i, n=sp["n"], fs=sp["fs"], a=sp["a"], floor=sp["floor"], K=sp["K"], rseed=rseed,
                columns=cols, logdet=osg.logdet, chi2=chi.tolist(), logL=ll.tolist(),
                r_checksum=[float(np.sum(sub[j].astype(np.float64))) for j in range(len(cols))])


def serving_checked():
    """The serving workload's first gapped N=8192 and first gapped N=16384
    segments: oracle logL of every column of their request pools (a request of
    K columns on a segment takes the pool's first K columns)."""
    fleet = inputs.serving_fleet()
    out = []
    for n in (8192, 16384):
        sp = next(x for x in fleet if x["n"] == n and x["gaps"] > 0)
        pool = inputs.serving_pool(n)
        kept = inputs.kept_index(sp["mask"], n)
        R = np.ascontiguousarray(pool[:, kept])
        osg = oracle.OracleSegment(inputs.acf_from_psd(n, sp["fs"]), sp["mask"])
        chi = osg.chi2(R)
        ll = oracle.loglike_from_chi2(chi, osg.logdet, osg.n_kept)
        out.append(dict(index=sp["index"], n=n, gaps=sp["gaps"], n_kept=osg.n_kept, logdet=osg.logdet,
                        logL=ll.tolist(), r_checksum=float(np.sum(R[:8].astype(np.float64)))))
    return out


def main():
    t0 = time.time()
    keys = sys.argv[1:]
    out = {}
    if keys and os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    want = (lambda k: not keys or k in keys)
    if want("single_n1024"):
        c1 = inputs.SINGLE_N1024
        out["single_n1024"] = one(c1["n"], c1["fs"], c1["seed"], 1, c1["seed"] + 1, [0])
    if want("gapfree_n8192_k4096"):
        c2 = inputs.GAPFREE_N8192_K4096
        cols2 = sample_cols(c2["K"], [0, 1, 2, 3, 127, 128, 129, 1000, 2047, 2048, 3001, 4094, 4095])
        out["gapfree_n8192_k4096"] = one(c2["n"], c2["fs"], c2["seed"], c2["K"], c2["seed"] + 1, cols2)
    if want("gapped_n16384_3det"):
        c3 = inputs.GAPPED_N16384_3DET
        cols3 = sample_cols(c3["K"], [0, 1, 100, 511, 512, 1022, 1023])
        dets = []
        for d, sc in enumerate(c3["scales"]):
            dets.append(one(c3["n"], c3["fs"], c3["seed"] + 10 * d, c3["K"], c3["seed"] + 10 * d + 1, cols3,
                            n_gaps=c3["n_gaps"], gap_len=c3["gap_len"], scale=sc))
        out["gapped_n16384_3det"] = dict(detectors=dets, columns=cols3,
                           joint_logL=np.sum([d_["logL"] for d_ in dets], axis=0).tolist())
    if want("mix64_longest"):
        out["mix64_longest"] = mix64_longest()
    if want("serving_checked"):
        out["serving_checked"] = serving_checked()
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
