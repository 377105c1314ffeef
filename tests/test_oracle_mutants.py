"""The oracle's pins bite: each plausible mistake, planted in a copy of the oracle
(on the CPU), makes the pins of its part fail (tests/test_oracle_pins.py for the
population likelihood, test_gridvt_pins.py for the grid selection term,
test_cbc_pins.py for the single-event CBC likelihood, test_grad_pins.py for the
gradient)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pop_oracle.c")

MUTANTS = {
    "power-law sign": ("pow(x, -alpha)", "pow(x, alpha)"),
    "gaussian exponent sign": ("exp(-0.5 * (x - mu)", "exp(0.5 * (x - mu)"),
    "truncation interval": ("erf((a - mu) / (SQRT2 * sigma))", "erf((0.0 - mu) / (SQRT2 * sigma))"),
    "mixture weight": ("(1.0 - lam) * pl + lam * pp", "(1.0 - lam) * pl + pp"),
    "mass-ratio exponent": ("(1.0 + beta) * pow(q, beta)", "(1.0 + beta) * pow(q, beta + 1.0)"),
    "mass-ratio normalisation": ("-expm1((1.0 + beta) * ln_ratio)", "-expm1(beta * ln_ratio)"),
    "beta exponent": ("pow(1.0 - a, bc - 1.0)", "pow(1.0 - a, bc)"),
    "isotropic tilt constant": ("(1.0 - xit) / 4.0", "(1.0 - xit) / 2.0"),
    "tilt truncation": ("truncnorm_pdf(c1, 1.0, sig, -1.0, 1.0)", "truncnorm_pdf(c1, 1.0, sig, -1.0, 3.0)"),
    "redshift end weights": ("(k == 0 || k == n - 1) ? 0.5 * f : f", "f"),
    "lower mass edge": ("if (!(m1 > mmin && m1 <= mmax))", "if (!(m1 >= mmin && m1 <= mmax))"),
    "q support": ("if (!(q * m1 >= mmin && q <= 1.0))", "if (!(q >= mmin / m1 && q < 1.0))"),
    "selection count": ("double xi = sw / (double)n_draw;", "double xi = sw / (double)(n_draw + n_found);"),
    "N factor of ln xi": ("sum_ln - (double)n_events * lnxi", "sum_ln - lnxi"),
    "event mean": ("log(s / (double)n_i)", "log(s)"),
    "prior weight": ("/ prior[j];", "* prior[j];"),
    "effective sample count": ("neff = var > 0.0 ? xi * xi / var", "neff = var > 0.0 ? 2.0 * xi * xi / var"),
    "variance of the mean": ("- xi * xi / (double)n_draw;", "- xi * xi / (double)n_found;"),
    "low-N_eff threshold": ("if (neff < 4.0 * (double)n_events)", "if (neff < 1.0 * (double)n_events)"),
}
GRID_MUTANTS = {
    "grid m1 weights": ("double wa = 0.5 * (", "double wa = ("),
    "grid q weights": ("double wq = 0.5 * (", "double wq = 0.25 * ("),
    "grid pdet transposed": ("pdet[(int64_t)a * n_q + b]", "pdet[(int64_t)b * n_m1 + a]"),
}
CBC_MUTANTS = {
    "cbc time-shift sign": ("const double ere = cos(ang), eim = -sin(ang);",
                            "const double ere = cos(ang), eim = sin(ang);"),
    "cbc 2/T": ("const double two_over_T = 2.0 * df;", "const double two_over_T = df;"),
    "cbc psd log term": ("-log(two_pi * S)", "-log(S)"),
    "cbc complex product": ("const double vim = cre * uim + cim * ure;", "const double vim = cre * uim - cim * ure;"),
    "cbc detector index": ("const double S = psd[(int64_t)i * M + j];", "const double S = psd[(int64_t)j * n_det + i];"),
    "cbc cross polarisation": ("Fc * hc[2 * j]", "Fp * hc[2 * j]"),
}
GRAD_MUTANTS = {
    "grad power-law normalisation": ("g[P_ALPHA] += fpl * (-log(m1) + dlnC_alpha);", "g[P_ALPHA] += fpl * (-log(m1));"),
    "grad upper edge sign": ("g[P_MMAX] += -fpl * plb - fnt * ntb;", "g[P_MMAX] += fpl * plb - fnt * ntb;"),
    "grad spin digamma factor": ("- 2.0 * pop_oracle_digamma(ac) + 2.0 * psab;", "- pop_oracle_digamma(ac) + psab;"),
    "grad tilt truncation": ("4.0 * std_normal_pdf(2.0 / sigt)", "2.0 * std_normal_pdf(2.0 / sigt)"),
    "grad selection term": ("G[p] = -(double)n_events * swg[p] / sw;", "G[p] = -swg[p] / sw;"),
}
PIN_FILES = {**{k: "test_oracle_pins.py" for k in MUTANTS}, **{k: "test_gridvt_pins.py" for k in GRID_MUTANTS},
             **{k: "test_cbc_pins.py" for k in CBC_MUTANTS}, **{k: "test_grad_pins.py" for k in GRAD_MUTANTS}}
ALL = {**MUTANTS, **GRID_MUTANTS, **CBC_MUTANTS, **GRAD_MUTANTS}


@pytest.mark.parametrize("name", sorted(ALL))
def test_pins_catch_mutant(name, tmp_path):
    old, new = ALL[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", str(mutant), "-o", str(lib), "-lm"],
                   check=True, capture_output=True)
    env = dict(os.environ, POP_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", PIN_FILES[name])],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant '{name}' survived the pins:\n{r.stdout[-2000:]}"
