"""The oracle's pins bite: each plausible mistake, planted in a copy of the oracle
(on the CPU), makes tests/test_oracle_pins.py fail."""
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
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", str(mutant), "-o", str(lib), "-lm"],
                   check=True, capture_output=True)
    env = dict(os.environ, POP_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant '{name}' survived the pins:\n{r.stdout[-2000:]}"
