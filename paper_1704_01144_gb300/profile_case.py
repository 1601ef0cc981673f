"""A fixed small case for profilers: W warm-up cycles, then one cycle.

    python -m paper_1704_01144_gb300.profile_case KIND N PREC W

KIND: ``ground`` (the ground-plane blast recipe, L = 6) or ``blast`` (the
graded spherical blast, L = 4); N: cubes per side of the mesh; PREC: 0 plain
FP64, 1 FP32-flux mode; W: warm-up cycles.  Prints one line with the mesh,
the launch configuration and the last cycle's face evaluations and cell
updates, the units the per-unit DRAM figures under ``profiles/`` divide by.
Under ncu, the launches of the last cycle follow those of the W warm-up
cycles (95 phases x 3 kernels + 2 local-step kernels per cycle at L = 6 in
the FP32-flux mode), which is what the ``-s`` and ``-c`` counts there
select.
"""
import sys

import torch

from . import build, fv, inputs as I


def main(argv):
    build.build()
    kind = argv[0] if len(argv) > 0 else "ground"
    n = int(argv[1]) if len(argv) > 1 else 80
    prec = int(argv[2]) if len(argv) > 2 else 1
    warm = int(argv[3]) if len(argv) > 3 else 1
    if kind == "ground":
        mesh, prim = I.ground_blast_case(n=n)
        L = 6
    elif kind == "blast":
        mesh, prim = I.blast_case(n=n, ratio=8.0)
        L = 4
    else:
        raise SystemExit(f"unknown case {kind!r} (ground or blast)")
    g = fv.Mesh(mesh, max_levels=L, precision=prec)
    g.set_state(prim)
    s = torch.cuda.Stream()
    g.advance(warm, stream=s, want_time=False)
    torch.cuda.synchronize()
    c0 = g.work_counters()
    g.advance(1, stream=s, want_time=False)
    torch.cuda.synchronize()
    c1 = g.work_counters()
    if g.status() != 0:
        raise SystemExit(fv.fv_last_error())
    print(f"case {kind} n={n} tets={g.n} faces={g.nf} L={L} prec={prec} launch={g.get_launch()} "
          f"cycle face_evals={c1[2] - c0[2]} cell_updates={c1[1] - c0[1]}")


if __name__ == "__main__":
    main(sys.argv[1:])
