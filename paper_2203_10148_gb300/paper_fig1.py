"""Re-run of the Sec. 4 experiments (the analogue of Fig. 1) on the GPU path.

For each test problem of eq. (9) (diffusion, diffusion-reaction,
advection-diffusion-reaction; `inputs.paper_pde`), discretised by P1 finite
elements as in Sec. 4 (`--discretization fem`, the default) or by finite
differences (`fd`), and N = 2^2 .. 2^6 slices,
PiTSBiCG (Algorithm 1) and parareal (eq. (6)) are run in FP64 from the same
initial guess (the coarse prediction G^{-1} B) and the preconditioned
residual ||G^{-1}(B - F X)||_{N,inf} is recorded against iterations and
against applications of G^{-1}F (matvecs: 2 per PiTSBiCG iteration, 1 per
parareal iteration, plus the initial residual for both).

    python -m paper_2203_10148_gb300.paper_fig1 [--n 49] [--N 4 8 16 32 64]
        [--discretization fem|fd] [--json FILE]

prints, per problem and N, the iterations and matvecs each method needs to
reduce the residual by --drop (default 1e-8).
"""
from __future__ import annotations

import argparse
import json
import sys
from typing import Dict, List, Optional

from . import inputs, pit


def run(pde: str, N: int, n: int = 49, max_iter: Optional[int] = None,
        discretization: str = "fem") -> Dict:
    """Residual histories of both methods for one problem and slice count."""
    w = inputs.paper_pde(pde, n=n, N=N, discretization=discretization)
    kmax = max_iter if max_iter is not None else N + 2
    with pit.Problem(w, "fp64") as p:
        _, info = p.bicgstab_solve(tol=1e-14, max_iter=kmax, history_len=kmax + 2)
        bicg = list(info[0]["history"])
        par: List[float] = []
        for k in range(0, min(kmax, N) + 1):
            _, pinfo = p.parareal_solve(kmax=k, tol=0.0)
            if k == 0:
                par.append(pinfo[0]["r0"])
            par.append(pinfo[0]["precond_resid"])
            if par[-1] <= 1e-14 * par[0]:
                break
    return {"pde": pde, "N": N, "n": n, "M": w.M, "fine_steps": w.fine[1],
            "discretization": discretization,
            "pitsbicg": {"residual": bicg, "matvecs": [1 + 2 * k for k in range(len(bicg))],
                         "status": info[0]["status_name"]},
            "parareal": {"residual": par[1:], "matvecs": [1 + k for k in range(len(par) - 1)]}}


def first_below(res: List[float], mv: List[int], drop: float):
    if not res:
        return None, None
    target = drop * res[0]
    for k, r in enumerate(res):
        if r <= target:
            return k, mv[k]
    return None, None


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=49, help="interior points per side (h = 1/(n+1))")
    ap.add_argument("--N", type=int, nargs="+", default=[4, 8, 16, 32, 64])
    ap.add_argument("--pde", nargs="+", default=list(inputs.PAPER_PDES))
    ap.add_argument("--drop", type=float, default=1e-8)
    ap.add_argument("--discretization", choices=["fem", "fd"], default="fem")
    ap.add_argument("--json", default=None, help="write the full histories here")
    args = ap.parse_args(argv)
    out = []
    print(f"| problem | N | PiTSBiCG iterations | PiTSBiCG matvecs | parareal iterations | "
          f"parareal matvecs |  (residual drop {args.drop:g})")
    print("|---|---|---|---|---|---|")
    for pde in args.pde:
        for N in args.N:
            r = run(pde, N, n=args.n, discretization=args.discretization)
            out.append(r)
            bi, bm = first_below(r["pitsbicg"]["residual"], r["pitsbicg"]["matvecs"], args.drop)
            pi, pm = first_below(r["parareal"]["residual"], r["parareal"]["matvecs"], args.drop)
            print(f"| {pde} | {N} | {bi} | {bm} | {pi} | {pm} |", flush=True)
    if args.json:
        with open(args.json, "w") as f:
            json.dump(out, f)
    return 0


if __name__ == "__main__":
    sys.exit(main())
