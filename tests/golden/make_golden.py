"""Write tests/golden/oracle_tiny.json: a tiny seeded stream, its initial cores and the
FP64 oracle's reconstructions.  Calls only oracle/ (inputs from numpy's seeded RNG).
The paper prints no worked example (no numbers for a specific small input), so this
fixture guards the oracle's arithmetic against regressions; its values are the
oracle's own, checked independently by the pins in test_oracle_pins.py.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle.ttals_oracle import OnlineTTALS, clamp_ranks  # noqa: E402


def main():
    rng = np.random.default_rng(20260601)
    dims = [4, 3, 5]
    ranks = clamp_ranks(dims, [3, 4, 2])
    full = [1] + ranks
    cores = [rng.standard_normal((full[k], dims[k], full[k + 1])) for k in range(3)]
    g = rng.standard_normal(full[-1])
    xs = [rng.standard_normal(dims) for _ in range(4)]
    st = OnlineTTALS(dims, ranks, cores, g)
    xh = [st.step(x) for x in xs]
    out = dict(citation="Algorithm 1 (Online TT-ALS), FP64 oracle output; no paper-printed example exists",
               dims=dims, ranks=ranks, cores=[c.tolist() for c in cores], g=g.tolist(),
               slices=[x.tolist() for x in xs], xhat=[x.tolist() for x in xh],
               final_g=st.g.tolist())
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
