"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

  python tests/golden/make_golden.py

tiny_top20.txt: the 100 x 900 tiny workload (seed 0: 50 clusters of 20, d = 128,
noise norm 0.3), k1 = 26, k2 = 7, L = 2 (Algorithm 1, Sec. 3.3; sum aggregator and
alpha = 2, Sec. 4.1).  Per query: the first 20 gallery indices of the oracle's
final list and their cosine scores (%.15e), then the oracle's top-26 neighbour
list of that query vertex (Eq. 8).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rerank_oracle  # noqa: E402
from paper_2012_07620_gb300 import synthetic  # noqa: E402

TOP = 20


def main():
    w = synthetic.make_workload(synthetic.TINY)
    ref = rerank_oracle.rerank(w.xq, w.xg, k1=26, k2=7, layers=2, mode="dense")
    lines = ["# tiny workload (seed 0), k1=26 k2=7 L=2; written by tests/golden/make_golden.py from oracle/ only",
             "# per query: q | top-20 gallery indices | their scores | top-26 neighbour list of vertex q"]
    for q in range(len(w.xq)):
        idx = ref.idx[q, :TOP]
        sc = ref.s[q, idx]
        lines.append(f"{q} | {' '.join(map(str, idx))} | {' '.join('%.15e' % v for v in sc)} | "
                     f"{' '.join(map(str, ref.knn_idx[q]))}")
    with open(os.path.join(HERE, "tiny_top20.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
