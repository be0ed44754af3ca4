"""Small seeded problems shared by the parity tests (inputs only: no solver arithmetic).

Each case gives a domain, a BoxArray, boundary conditions, scalars and dense fields
(alpha, beta, rhs) from a seeded generator.  Sizes are chosen so the oracle finishes in
seconds while spanning several boxes, uneven box sizes (ragged tails) and both
coarsening paths (per box, then aggregation into one box).
"""
import numpy as np

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def dom3(nx, ny, nz):
    return ((0, 0, 0), (nx - 1, ny - 1, nz - 1))


def make(name):
    if name == "poisson32":
        c = I.poisson32()
        c["prob_hi"] = (1.0, 1.0, 1.0)
        return c
    rng = np.random.default_rng(SEEDS[name])
    if name == "uneven":  # 20x12x14 in boxes of <= 6: tails of 2, aggregation to a 10x6x7 bottom
        n = (20, 12, 14)
        bc_lo = bc_hi = [D_] * 3
        a, b, mgs = 0.0, 1.0, 6
    elif name == "periodic":  # singular: all periodic, a = 0
        n = (16, 12, 8)
        bc_lo = bc_hi = [P_] * 3
        a, b, mgs = 0.0, 1.0, 8
    elif name == "helmholtz":  # x periodic, y/z walls, a*alpha term, b != 1, anisotropic h
        n = (16, 16, 16)
        bc_lo = bc_hi = [P_, D_, D_]
        a, b, mgs = 1.5, 2.0, 8
    elif name == "oddlo":  # boxes of 5: nothing coarsens, the whole level is the bottom
        n = (10, 10, 10)
        bc_lo = bc_hi = [D_] * 3
        a, b, mgs = 0.0, 1.0, 5
    elif name == "abec64":  # the abec256 recipe at 64^3 in 16^3 boxes
        n = (64, 64, 64)
        bc_lo = bc_hi = [D_] * 3
        a, b, mgs = 0.0, 1.0, 16
    elif name == "neumann":  # singular: zero-flux walls everywhere, a = 0; tails of 4
        n = (20, 16, 12)
        bc_lo = bc_hi = [N_] * 3
        a, b, mgs = 0.0, 1.0, 8
    elif name == "mixedwalls":  # Neumann/Dirichlet per side, y periodic, a*alpha term, anisotropic h
        n = (24, 16, 20)
        bc_lo, bc_hi = [N_, P_, D_], [D_, P_, N_]
        a, b, mgs = 0.5, 1.3, 6
    else:
        raise KeyError(name)
    shape = (n[2], n[1], n[0])
    dom = dom3(*n)
    beta = I.lognormal_beta(rng, shape, periodic=(bc_lo[0] == P_ and bc_lo[1] == P_))
    alpha = np.exp(rng.standard_normal(shape)) if a != 0.0 else None
    rhs = rng.standard_normal(shape)
    if D_ not in bc_lo + bc_hi and a == 0.0:  # singular: a zero-mean rhs
        rhs -= rhs.mean()
    prob_hi = {"helmholtz": (1.0, 0.5, 2.0), "mixedwalls": (1.2, 0.8, 1.0)}.get(name, (1.0, 1.0, 1.0))
    return dict(name=name, domain=dom, boxes=I.chop(*dom, mgs), bc_lo=list(bc_lo), bc_hi=list(bc_hi), a=a, b=b,
                alpha=alpha, beta=beta, rhs=rhs, prob_hi=prob_hi)


SEEDS = {"uneven": 101, "periodic": 102, "helmholtz": 103, "oddlo": 104, "abec64": 105, "neumann": 106,
         "mixedwalls": 107}
NAMES = ["uneven", "periodic", "helmholtz", "oddlo", "poisson32", "neumann", "mixedwalls"]
