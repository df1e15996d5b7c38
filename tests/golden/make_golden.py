"""Write the stored oracle values under tests/golden/.

    python tests/golden/make_golden.py

The paper prints no worked example (its result figures are placeholders), so
nothing here is the paper's number. These files hold the FP64 oracle's results
on small seeded chains, written by this script, which calls only ``oracle`` and
the seeded input generator (``paper_1609_06779_gb300.synth``, which holds none
of the method's arithmetic). They make a later change to the oracle's
arithmetic show up as a diff (CPU test) and give the GPU tests fixed values to
meet without running the oracle. The oracle itself is pinned independently by
``tests/test_oracle_pins.py`` (closed forms, dense definitions, conservation).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1609_06779_gb300 import synth  # noqa: E402

# name -> (chain lengths, model seed, state seed): single links, the two-link
# arm's size, the 7-link chain of the shared-model batch, a 32-link chain of the
# uniform batch, and a ragged 33-link chain (one past a power of two for OEE)
CASES = {
    "fd_small_chains": ([1, 2, 7, 32, 33], 5, 6),
}


def case_values(lengths, model_seed, state_seed):
    model = synth.random_chains(lengths, seed=model_seed)
    st = synth.random_states(model.n_links_total, seed=state_seed)
    qdd_in = np.random.default_rng(state_seed + 1).standard_normal(model.n_links_total)
    return {
        "source": "FP64 oracle (oracle/fd_oracle.c) on synth.random_chains(lengths, "
                  "seed=model_seed) and synth.random_states(n_links, seed=state_seed); "
                  "qdd_in = default_rng(state_seed + 1).standard_normal(n_links)",
        "lengths": list(lengths), "model_seed": model_seed, "state_seed": state_seed,
        # forward dynamics, Eq. 4 (dense Cholesky of M), ABIA (Section II-C, the
        # ABA route) and CFA with odd-even elimination (Algorithms 1 and 2)
        "qdd_cholesky": oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky").tolist(),
        "qdd_aba": oracle.fd(model, st.q, st.qdot, st.tau, algo="aba").tolist(),
        "qdd_cfa": oracle.fd(model, st.q, st.qdot, st.tau, algo="cfa").tolist(),
        # inverse dynamics, Eq. 2a-2d, at (q, qdot, qdd_in)
        "tau_id": oracle.rnea_batch(model, st.q, st.qdot, qdd_in).tolist(),
    }


def main():
    for name, (lengths, ms, ss) in CASES.items():
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(case_values(lengths, ms, ss), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
