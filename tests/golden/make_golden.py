"""Write tests/golden/oracle_water300.json from the FP64 oracle alone.

A regression fixture: it pins the oracle against its own earlier output (any
change to the oracle's arithmetic must be deliberate and must regenerate this
file in the same commit, naming the passage of the paper that justifies it).
It calls only ``oracle`` and the seeded input generator.

    python tests/golden/make_golden.py
"""
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1309_1889_gb300 import inputs  # noqa: E402


def main():
    cfg = dict(n_atoms=300, region=1.5, margin=0.5, a=1.2, h=0.25, levels=3)
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=cfg["margin"], with_velocities=False)
    m = oracle.msm(s.pos, s.q, s.box, cfg["a"], cfg["h"], cfg["levels"])
    rows = [0, 1, 2, 57, 158, 299]
    cfg.update(energy=m["energy"], force_rows=rows, forces=m["forces"][rows].tolist(),
               source="oracle.msm (FP64, msm_oracle.c)")
    out = Path(__file__).resolve().parent / "oracle_water300.json"
    out.write_text(json.dumps(cfg, indent=1) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
