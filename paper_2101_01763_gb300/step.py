"""Run whole steps (spand_factor + sstep_gmres_solve) of one seeded workload,
for profilers: no timing, no reference, nothing but the library's launches
after assembly.

    python -m paper_2101_01763_gb300.step [--config C2] [--precision mixed] [--steps 2]
"""
import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="C2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=2)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    import paper_2101_01763_gb300 as sg
    from synth import get_config, modal_state, naca_ogrid
    c = get_config(a.config)
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    dev = torch.device("cuda")
    rhs, A, _ = sg.assemble(torch.as_tensor(X, device=dev), c.p, torch.as_tensor(u, device=dev), c.mach,
                            c.alpha_deg, c.cfl)
    plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
    for _ in range(a.steps):
        F = sg.Factor(plan, A, c.eps, a.precision)
        x, st = sg.sstep_gmres(A, F, rhs, s=c.s, restart=c.restart, tol=c.tol, max_iters=c.max_iters)
        torch.cuda.synchronize()
        F.close()
    print(f"{a.config} {a.precision}: {a.steps} steps, last solve {st['iters']} iterations, "
          f"relres {st['true_relres']:.2e}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
