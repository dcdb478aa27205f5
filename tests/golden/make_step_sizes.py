"""Write tests/golden/opnorm_full_mask.txt: L = ||K||_2 of the full-mask operator
(pseudocode step 1 of Sec. II.A) for each slice size, from the FP64 oracle's
power iteration.  Calls only oracle/; run from the repository root:

    python tests/golden/make_step_sizes.py
"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import pd_oracle as O  # noqa: E402

SIZES = [(64, 64, 0), (64, 64, 1), (128, 128, 0), (192, 192, 0), (256, 256, 0), (384, 384, 0), (512, 512, 0)]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "opnorm_full_mask.txt")
    lines = [
        "# L = ||K||_2, K = [W D; M G] with W = M = 1 (full mask), by the FP64 oracle's power",
        "# iteration (rtol 1e-12); written by tests/golden/make_step_sizes.py.",
        "# columns: H W b0_axis L",
    ]
    for H, W, ax in SIZES:
        L = O.opnorm(np.ones((H, W)), b0_axis=ax)
        lines.append(f"{H} {W} {ax} {L:.15f}")
        print(lines[-1], flush=True)
    open(out, "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
