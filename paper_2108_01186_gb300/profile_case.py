"""Small, self-contained workloads for profiling captures (none uses the oracle).

Default case: one system of n^3 points (spacing 0.2 bohr) with `norb` Gaussian
orbital densities (no randomness), solved once by the library's multigrid-
preconditioned CG or Kronecker solver (mixed precision by default).  Small
enough for an ncu --set full capture of one stencil launch (8 x 128^3 float32
vectors: 64 MiB each, above L2).  The flo and step cases use the seeded
synthetic systems of the benchmark's recipe.

  python -m paper_2108_01186_gb300.profile_case --n 128 --norb 8 [--fp64] [--solver kron]
  python -m paper_2108_01186_gb300.profile_case --case flo     (FLO build, 96^3, 16+16 orbitals)
  python -m paper_2108_01186_gb300.profile_case --case step --norb 12   (forward + adjoint, n^3, 12+12)
"""
import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--norb", type=int, default=8)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--solver", default="pcg", choices=["pcg", "kron"],
                    help="inner solver of the mixed refinement (kron: the Kronecker-product transforms)")
    ap.add_argument("--case", default="poisson", choices=["poisson", "flo", "step"],
                    help="poisson: one multigrid-PCG solve of Gaussian densities; flo: two FLO builds "
                         "(tensor-core overlap) of the seeded 96^3, 16+16-orbital system; step: one "
                         "forward + adjoint step (Kronecker solver) of a seeded n^3 system "
                         "(spacing 0.2 bohr) with norb + norb orbitals")
    args = ap.parse_args()
    if args.case == "flo":
        return flo_case(args)
    if args.case == "step":
        return step_case(args)
    import torch
    from paper_2108_01186_gb300 import build
    from paper_2108_01186_gb300.flosic import Context

    build.build()
    n, N, h = args.n, args.norb, 0.2
    o = -0.5 * h * (n - 1)
    ctx = Context([dict(n=n, h=h, origin=[o, o, o], norb=[N])], precision=0 if args.fp64 else 1,
                  cg_tol=1e-10, preconditioner=1, solver=2 if args.solver == "kron" else 0)
    x = torch.linspace(o, -o, n, dtype=torch.float64, device="cuda")
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    phi = torch.cat([torch.exp(-(X - 0.3 * k) ** 2 - Y ** 2 - Z ** 2).reshape(-1) for k in range(N)]).contiguous()
    V, it, conv = ctx.orbital_poisson(phi)
    torch.cuda.synchronize()
    print("iterations", it.tolist(), "converged", conv.tolist())


def flo_case(args):
    import numpy as np
    import torch
    from paper_2108_01186_gb300 import build, synth
    from paper_2108_01186_gb300.flosic import Context

    build.build()
    s = synth.make_config(1)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi]), device="cuda")
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods]), device="cuda")
    ctx = Context([s], precision=0 if args.fp64 else 1, cg_tol=1e-10)
    for _ in range(2):
        phi, S, Q = ctx.build_flos(psi, fods)
    torch.cuda.synchronize()
    print("sum of S", float(S.double().sum()))


def step_case(args):
    import numpy as np
    import torch
    from paper_2108_01186_gb300 import build, synth
    from paper_2108_01186_gb300.flosic import Context

    build.build()
    s = synth.make_system(args.n, 0.2, 8, [args.norb, args.norb], seed=77)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi]), device="cuda")
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods]), device="cuda")
    ctx = Context([s], precision=1, cg_tol=1e-10, solver=2)
    out = ctx.forward(psi, fods)
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    dpsi, dfod = ctx.sic_backward(psi, fods, out["phi"], out["V"], gE)
    torch.cuda.synchronize()
    print("E_sic", float(out["E_sic"][0]), "max |dE/da|", float(dfod.abs().max()))


if __name__ == "__main__":
    main()
