"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a private copy of the oracle source (a
flipped sign, a transposed operand, a dropped term, a wrong index or
comparison), compiles it on the CPU and runs the pin suites (method and
gradient) against it in a child process: the suites must fail.  The real oracle is never modified.
"""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pmmf_oracle.c")

MUTANTS = [
    ("transposed Givens block",
     "O[0] = c; O[1] = -s; O[2] = s; O[3] = c;",
     "O[0] = c; O[1] = s; O[2] = -s; O[3] = c;"),
    ("Gram uses one row twice",
     "acc = fma(val[pa], val[pb], acc);",
     "acc = fma(val[pa], val[pa], acc);"),
    ("eliminates the larger off-diagonal norm",
     "if (d <= dbest) { dbest = d; bi = a; }",
     "if (d >= dbest) { dbest = d; bi = a; }"),
    ("residual drops the active-row terms",
     "                            contrib = contrib + w->val[e2] * w->val[e2];\n                        } else {",
     "                        } else {"),
    ("inverse sweep uses untransposed blocks",
     "for (int b = 0; b < kk; ++b) Ot[a * kk + b] = O[b * kk + a];",
     "for (int b = 0; b < kk; ++b) Ot[a * kk + b] = O[a * kk + b];"),
    ("Jacobi sign of the angle flipped",
     "*s = (h >= 0.0 ? g : -g) / den;",
     "*s = (h >= 0.0 ? -g : g) / den;"),
    ("Jacobi drops the coupling from the root",
     "double r = sqrt(h * h + g * g);",
     "double r = sqrt(h * h);"),
    ("symmetric update forgets the column mirror",
     "            X[y * ld + T[a]] = out[a];\n",
     ""),
    ("clustering distance ignores the last dimension",
     "for (int d = 0; d < dim; ++d) {\n        int64_t t = (int64_t)q[d] - c[d];",
     "for (int d = 0; d + 1 < dim; ++d) {\n        int64_t t = (int64_t)q[d] - c[d];"),
    ("partner score not normalised",
     "double sc = fabs(G[i * cu + j]) * w;",
     "double sc = fabs(G[i * cu + j]);"),
    ("H keeps the wrong diagonal",
     "if (w->col[e2] == x) f->hdiag[x] = w->val[e2];",
     "if (w->col[e2] == x) f->hdiag[x] = 0.0;"),
    ("gradient drops the transposed occurrence of each block",
     "dq[e * kk + c] = dq[e * kk + c] + ga[c] * pin[(q * K + e) * nrhs + r];",
     "dq[e * kk + c] = dq[e * kk + c];"),
    ("gradient of a block entry transposed",
     "dq[c * kk + e] = dq[c * kk + e] + gb[c] * vin[(q * K + e) * nrhs + r];",
     "dq[e * kk + c] = dq[e * kk + c] + gb[c] * vin[(q * K + e) * nrhs + r];"),
    ("angle chain rule with a flipped sine term",
     "dtheta[q] = -s * (dq[0] + dq[3]) + c * (dq[2] - dq[1]);",
     "dtheta[q] = -s * (dq[0] + dq[3]) + c * (dq[1] - dq[2]);"),
    ("inverse square root divides the wavelets by H_xx",
     "z[x * nrhs + r] = inverse == 2 ? z[x * nrhs + r] / sqrt(f->hdiag[x])",
     "z[x * nrhs + r] = inverse == 2 ? z[x * nrhs + r] / f->hdiag[x]"),
    ("core inverse square root without the square root",
     "acc = acc + V[a * m + i] * V[a * m + j] / sqrt(w[a]);",
     "acc = acc + V[a * m + i] * V[a * m + j] / w[a];"),
    ("split CG returns y instead of W y",
     "    st = or_apply(f, OR_OP_A_INV_SQRT, y, x, nrhs);         /* x = W y */",
     "    memcpy(x, y, sz);"),
    ("split CG applies W on one side only",
     "        st = or_apply(f, OR_OP_A_INV_SQRT, qv, qv, nrhs);\n",
     ""),
    ("block angles taken from the transposed entries",
     "            const double t = atan2(A[l * kk + j], A[j * kk + j]);",
     "            const double t = atan2(A[j * kk + l], A[j * kk + j]);"),
    ("angle chain rule with the derivative's sine sign flipped",
     "acc = acc + Lam[j * kk + b] * (-s * bj - c * bl) + Lam[l * kk + b] * (c * bj - s * bl);",
     "acc = acc + Lam[j * kk + b] * (s * bj - c * bl) + Lam[l * kk + b] * (c * bj - s * bl);"),
    ("inverse gradient of H without the minus sign",
     "                dhdiag[i] = -acc;",
     "                dhdiag[i] = acc;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not found exactly once"
    mdir = tmp_path / "oracle"
    mdir.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "pmmf_oracle.h"), mdir)
    (mdir / "pmmf_oracle.c").write_text(src.replace(old, new))
    so = str(mdir / "libmutant.so")
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-w", "-o", so, str(mdir / "pmmf_oracle.c"), "-lm"])
    env = dict(os.environ, PMMF_ORACLE_SO=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_grad_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant '{name}' survived the pins:\n{r.stdout[-2000:]}"
