"""Writes chip_embed3h_failure.json: the oracle's outcome of the full-size orthogonal-cutting
block (4 x 1 x 0.4 mm, h = 1/68 mm, Ti-6Al-4V Johnson-Cook, Sec. 4.2) with the rigid tool
embedded 3 h into the work piece. The contact projection of the first step (Sec. 3.3) drives a
material point outside the convex hull of its new support, where the LME problem of Sec. 2.2
has no finite minimiser; the oracle reports the status and the ID of the first such point.

Runs the oracle only (about 3 minutes and 30 GB of host memory): python tests/golden/make_chip_embedding_failure.py"""
import json
import pathlib
import sys

HERE = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parent.parent))

import oracle  # noqa: E402
import scenarios  # noqa: E402

EMBED_H = 3.0
STEPS = 2


def main():
    h = 1.0e-3 / 68
    p = scenarios.chip_block(h=h, embed=EMBED_H * h, steps=STEPS)
    sim = oracle.Sim(p)
    st = sim.step(STEPS)
    c = sim.counts()
    out = dict(embed_h=EMBED_H, steps=STEPS, status=int(st), mp_id=int(c["err_id"]), step_reached=int(c["step"]),
               n_nodes=p.n_nodes, n_mps=p.n_mps,
               source="oracle.Sim on scenarios.chip_block(h=1/68 mm, embed=3 h), written by make_chip_embedding_failure.py")
    (HERE / "chip_embed3h_failure.json").write_text(json.dumps(out, indent=1) + "\n")
    print(out)


if __name__ == "__main__":
    main()
