"""Write tests/golden/tiny_oracle.json from the FP64 oracle only.

The paper prints no worked example with numbers for any object (its only
printed constant on this path is the 0.8 GeV stub threshold, Section 2), so
the stored values here are the oracle's own output on the seeded tiny
workload. They guard the oracle against unintended changes; any change to
them must come with a commit that names the passage or reading behind it.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O            # noqa: E402
from synth import events as E, geometry as G, maps as M   # noqa: E402
from synth.config import DEFAULT_CUTS     # noqa: E402


def snapshot(seed):
    g = G.make_geometry(barrel_only=True)
    ev = E.tiny_event(seed, g)
    r = O.Setup(g.module_table(), M.load_maps(g), DEFAULT_CUTS, ev).run()
    tcs = []
    for i in range(r["tc"]["n"]):
        hs = sorted(int(r["tc"][f"h{j}"][i]) for j in range(10) if r["tc"][f"h{j}"][i] >= 0)
        tcs.append([int(r["tc"]["type"][i]), int(r["tc"]["seed"][i]), hs])
    return dict(counts={k: int(r[k]["n"]) for k in O.STAGES}, tc=sorted(tcs))


if __name__ == "__main__":
    out = {"workload": "tiny barrel event, 10 tracks + 20 noise hits", "seeds": {}}
    for s in range(3):
        out["seeds"][str(s)] = snapshot(s)
    with open(os.path.join(HERE, "tiny_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
