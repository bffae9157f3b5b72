"""Writes one_voxel_posteriors.txt: the occupancy posterior of one voxel seen
by K cameras whose likelihood maps hold s_1 .. s_K at the voxel's pixel, in
exact rational arithmetic.

The posterior is the product form of Eq. 3-4 over the cameras, with each
camera's two likelihoods from Eq. 5 marginalised over occlusion with
P(O) = 1/2 under detection rate P_D and false-alarm rate P_FA:
    a = P_D s + (1 - P_D)(1 - s)           (voxel occupied)
    f = P_FA s + (1 - P_FA)(1 - s)         (nothing on the viewing line)
    b = (f + a) / 2                        (voxel empty)
    occ = prior prod(a) / (prior prod(a) + (1 - prior) prod(b)).
With P_D = 1 and P_FA = 0 this is Eq. 6-9 as printed.  Uses only the
standard library (fractions): no value comes from the oracle or the GPU
path.  Run from the repository root:  python tests/golden/make_one_voxel_posteriors.py

It also writes one_voxel_adjoint.txt: for the same cases with every a > 0,
d occ / d s_k = occ (1 - occ) (a_k' / a_k - b_k' / b_k), the derivative of
that posterior with respect to camera k's SLM value, where a' = 2 P_D - 1
and b' = (a' + f') / 2 with f' = 2 P_FA - 1 (the chain rule through the
log-odds; its derivation is the quotient rule on occ).
"""
import os
from decimal import Decimal, localcontext
from fractions import Fraction as Fr

RATES = [("1", "0", "1/2"), ("9/10", "1/10", "1/2"), ("4/5", "3/10", "1/5"), ("7/10", "1/20", "2/3"),
         ("3/5", "2/5", "9/10")]
# dyadic SLM values (exact in binary floating point)
SLMS = [["1/4"], ["3/4", "1/2"], ["1", "1/8", "5/8"], ["0", "1/2", "1", "3/4"], ["7/8"] * 6,
        ["1/16", "15/16", "3/8", "5/16", "1/2", "11/16", "1", "13/16"], ["1/2"] * 5]


def posterior(pd, pfa, prior, slms):
    num, den_b = prior, 1 - prior
    for s in slms:
        a = pd * s + (1 - pd) * (1 - s)
        f = pfa * s + (1 - pfa) * (1 - s)
        num *= a
        den_b *= (f + a) / 2
    return num / (num + den_b)


def decimal_of(q):
    """The exact rational q to 25 significant digits."""
    with localcontext() as ctx:
        ctx.prec = 25
        return str(Decimal(q.numerator) / Decimal(q.denominator))


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "one_voxel_posteriors.txt")
    lines = ["# One voxel, K cameras: exact posterior of the product form of Eq. 3-4 with Eq. 5's",
             "# occlusion marginalisation (P(O) = 1/2); P_D = 1, P_FA = 0 is Eq. 6-9.",
             "# Written by make_one_voxel_posteriors.py (exact rationals).",
             "# columns: p_detect p_false_alarm prior s_1,...,s_K occupancy (25 significant digits)"]
    for pd, pfa, prior in RATES:
        for slms in SLMS:
            occ = posterior(Fr(pd), Fr(pfa), Fr(prior), [Fr(s) for s in slms])
            lines.append(f"{pd} {pfa} {prior} {','.join(slms)} {decimal_of(occ)}")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "one_voxel_adjoint.txt")
    lines = ["# One voxel, K cameras: exact d occ / d s_k of the posterior in one_voxel_posteriors.txt",
             "# (cases with every a > 0).  Written by make_one_voxel_posteriors.py (exact rationals).",
             "# columns: p_detect p_false_alarm prior s_1,...,s_K d_1,...,d_K (25 significant digits)"]
    for pd, pfa, prior in RATES:
        P_D, P_FA, PRIOR = Fr(pd), Fr(pfa), Fr(prior)
        for slms in SLMS:
            s_ = [Fr(s) for s in slms]
            a = [P_D * s + (1 - P_D) * (1 - s) for s in s_]
            if any(x == 0 for x in a):
                continue
            occ = posterior(P_D, P_FA, PRIOR, s_)
            da = 2 * P_D - 1
            db = (da + 2 * P_FA - 1) / 2
            b = [(P_FA * s + (1 - P_FA) * (1 - s) + ak) / 2 for s, ak in zip(s_, a)]
            d = [occ * (1 - occ) * (da / ak - db / bk) for ak, bk in zip(a, b)]
            lines.append(f"{pd} {pfa} {prior} {','.join(slms)} {','.join(decimal_of(x) for x in d)}")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
