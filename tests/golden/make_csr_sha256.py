#!/usr/bin/env python3
"""Write tests/golden/csr_sha256.txt: the SHA-256 of every workload's CSR and first source set.

Calls only the seeded input generators (paper_2103_14915_gb300.inputs); no
part of the query method runs. One line per workload:

    <workload> n=<n> m=<m> csr=<sha256> sources=<sha256>

csr hashes row_ptr (int64), col (int32) and, for weighted graphs, w (int32),
in that order, little-endian as the arrays hold them; sources hashes the
int32 ids of workload_sources(name, g) (set 0). A changed generator changes
these values, which tests/test_inputs.py and bench.py check.

    python tests/golden/make_csr_sha256.py [workload ...]
"""
from __future__ import annotations

import hashlib
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from paper_2103_14915_gb300 import inputs  # noqa: E402

OUT = Path(__file__).resolve().parent / "csr_sha256.txt"
WORKLOADS = ["rmat14_plain_sssp", "grid1024_bfs_sssp", "rmat22_ppr", "rmat24_sssp", "rmat25_serving"]


def csr_sha256(g) -> str:
    h = hashlib.sha256()
    h.update(g.row_ptr.astype("<i8", copy=False).tobytes())
    h.update(g.col.astype("<i4", copy=False).tobytes())
    if g.w is not None:
        h.update(g.w.astype("<i4", copy=False).tobytes())
    return h.hexdigest()


def sources_sha256(src) -> str:
    return hashlib.sha256(src.astype("<i4", copy=False).tobytes()).hexdigest()


def line(name: str) -> str:
    g = inputs.workload_graph(name)
    src = inputs.workload_sources(name, g)
    return f"{name} n={g.n} m={g.m} csr={csr_sha256(g)} sources={sources_sha256(src)}"


def read(path: Path = OUT) -> dict:
    """{workload: {"n": int, "m": int, "csr": hex, "sources": hex}} from the golden file."""
    out = {}
    for ln in path.read_text().splitlines():
        if not ln.strip() or ln.startswith("#"):
            continue
        name, *kv = ln.split()
        d = dict(x.split("=", 1) for x in kv)
        out[name] = {"n": int(d["n"]), "m": int(d["m"]), "csr": d["csr"], "sources": d["sources"]}
    return out


def main(names):
    have = read() if OUT.exists() else {}
    for name in names:
        ln = line(name)
        print(ln, flush=True)
        _, *kv = ln.split()
        d = dict(x.split("=", 1) for x in kv)
        have[name] = {"n": int(d["n"]), "m": int(d["m"]), "csr": d["csr"], "sources": d["sources"]}
    body = ["# SHA-256 of each workload's CSR (row_ptr i64, col i32[, w i32]) and source set 0 (i32).",
            "# Written by tests/golden/make_csr_sha256.py from the seeded generators only."]
    for name in WORKLOADS:
        if name in have:
            v = have[name]
            body.append(f"{name} n={v['n']} m={v['m']} csr={v['csr']} sources={v['sources']}")
    OUT.write_text("\n".join(body) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or WORKLOADS)
