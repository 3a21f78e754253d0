"""Writes ``tiny_joint.txt``: the oracle's ids and depths for a tiny joint
(foveated + rolling) frame.  Calls only the oracle; a regression fixture that
guards the oracle against unintended change (the paper prints no worked
numeric example of the method's output).

    python -m tests.golden.make_golden
"""
import os

import numpy as np

from paper_1806_05385_gb300 import scenes as S


def golden_case():
    sc = S.random_triangles(24, 123, vel_sigma=0.08, offset=0.5)
    p0, p1 = S.head_poses(3.0, 1.0, 0.032)
    view = S.View(W=20, H=14, tan_x=0.55, tan_y=0.4, pose0=p0, pose1=p1, mode=S.MODE_BOTH,
                  fovea=(0.4, 0.6), alpha=2.0)
    return view, sc


def main():
    from oracle import oracle as O
    view, sc = golden_case()
    o = O.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_joint.txt")
    with open(path, "w") as f:
        f.write("# oracle ids and ray parameters for golden_case() (20x14, joint mode)\n")
        f.write("# written by tests/golden/make_golden.py; columns: pixel id s\n")
        for n in range(o["id"].shape[0]):
            f.write(f"{n} {int(o['id'][n])} {float(o['s'][n])!r}\n")


if __name__ == "__main__":
    main()
