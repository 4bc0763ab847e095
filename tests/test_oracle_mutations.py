"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/kc_oracle.c (a dropped
term, a wrong sign, a transposed index, a wrong operand), compiles it on the
CPU, installs it in place of the real oracle and runs the pin suite of
tests/test_oracle.py against it: at least one pin has to fail.  The real
oracle is restored afterwards and must pass them all again.
"""
import inspect
import os

import pytest

import oracle
import test_oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "kc_oracle.c")

# (name, original text, mistaken text)
MUTATIONS = [
    ("M0 sign (Eq. 6 as printed)", "phase + M0 / KCO_TWO_PI", "phase - M0 / KCO_TWO_PI"),
    ("epoch ignored", "fmod(t - t0, P) / P", "fmod(t, P) / P"),
    ("Kepler sign", "double f = E - e * sin(E) - M;", "double f = E + e * sin(E) - M;"),
    ("true anomaly factors swapped",
     "sqrt(1.0 + e) * sin(0.5 * E), sqrt(1.0 - e) * cos(0.5 * E)",
     "sqrt(1.0 - e) * sin(0.5 * E), sqrt(1.0 + e) * cos(0.5 * E)"),
    ("e cos w term dropped", "return K * (cos(w + f) + e * cos(w));", "return K * (cos(w + f));"),
    ("sin for cos in e term", "return K * (cos(w + f) + e * cos(w));",
     "return K * (cos(w + f) + e * sin(w));"),
    ("gamma dropped", "double V = gamma, r;", "double V = 0.0, r;"),
    ("residual sign", "r = V - v[k];", "r = V + v[k];"),
    ("weight is 1/sigma", "double wk = 1.0 / var;", "double wk = 1.0 / sqrt(var);"),
    ("jitter not squared", "sigma[k] * sigma[k] + jitter * jitter",
     "sigma[k] * sigma[k] + jitter"),
    ("Neumaier compensation sign", "a->c += (a->s - t) + x;", "a->c += (a->s - t) - x;"),
    ("eccentricity range", "e >= 0.0 && e < 1.0", "e >= 0.0 && e <= 1.0"),
    ("dv/dK misses e cos w", "g[1] = c_wf + e * cos(w);", "g[1] = c_wf;"),
    ("dv/dw misses e sin w", "g[3] = -K * (s_wf + e * sin(w));", "g[3] = -K * s_wf;"),
    ("dv/de misses dE/de", "sin(E) / (beta * D) + df_dE * sin(E) / D", "sin(E) / (beta * D)"),
    ("dM/dP ignores the epoch", "(-KCO_TWO_PI * (t - t0) / (P * P))",
     "(-KCO_TWO_PI * t / (P * P))"),
    ("dM/dP sign", "(-KCO_TWO_PI * (t - t0) / (P * P))", "(KCO_TWO_PI * (t - t0) / (P * P))"),
    ("gradient index transposed", "kco_sum_add(&gsum[5 * j + q], a * g[j][q]);",
     "kco_sum_add(&gsum[5 * j + q], a * g[q % 5][j % 5]);"),
    ("dchi2/dgamma factor", "kco_sum_add(&gsum[5 * n_pl], a);",
     "kco_sum_add(&gsum[5 * n_pl], 0.5 * a);"),
    ("nll log term dropped", "0.5 * (wk * r * r + log(KCO_TWO_PI * var))", "0.5 * (wk * r * r)"),
    ("nll jitter gradient sign", "sj * wk * (1.0 - wk * r * r)", "sj * wk * (1.0 + wk * r * r)"),
    ("nll gradient factor", "double a = wk * r;", "double a = 2.0 * wk * r;"),
    ("DE-MC acceptance sign", "log(u[3 * c]) < -0.5 * (chi2_prop[c] - chi2[i])",
     "log(u[3 * c]) < 0.5 * (chi2_prop[c] - chi2[i])"),
    ("DE-MC gamma dropped", "proposals[c * n_par + p] = (xi + gamma * d) + eps;",
     "proposals[c * n_par + p] = (xi + d) + eps;"),
    ("DE-MC partners may coincide", "if (k2 >= k1) k2 += 1;", "if (k2 > k1) k2 += 1;"),
    ("DE-MC perturbation not relative", "double eps = (eps_scale[p] * fabs(xi)) * z[c * n_par + p];",
     "double eps = eps_scale[p] * z[c * n_par + p];"),
    ("Gauss-Newton weight dropped", "kco_sum_add(&acc[i++], wk * J[p] * J[q]);",
     "kco_sum_add(&acc[i++], J[p] * J[q]);"),
    ("Gauss-Newton index", "kco_sum_add(&acc[i++], wk * J[p] * J[q]);",
     "kco_sum_add(&acc[i++], wk * J[p] * J[p]);"),
    ("Gauss-Newton gamma column", "J[5 * n_pl] = 1.0;                                        /* dV/dgamma */",
     "J[5 * n_pl] = 0.0;"),
    ("prediction without gamma", "double V = par[5 * n_pl];\n            for (j = 0; j < n_pl; ++j) V +=",
     "double V = 0.0;\n            for (j = 0; j < n_pl; ++j) V +="),
]


def pin_tests():
    for name, fn in inspect.getmembers(test_oracle, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        params = inspect.signature(fn).parameters
        if "t0" in params:
            for t0 in (2450000.0, 0.0):
                yield f"{name}[{t0}]", (lambda fn=fn, t0=t0: fn(oracle, t0))
        else:
            yield name, (lambda fn=fn: fn(oracle))


def failing_pins():
    failed = []
    for name, run in pin_tests():
        try:
            run()
        except Exception:              # assertion or numerical error: the pin fired
            failed.append(name)
    return failed


@pytest.mark.parametrize("name,orig,bad", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, bad):
    src = open(SRC).read()
    assert orig in src, f"mutation anchor not found: {orig!r}"
    mutant = oracle.compile_variant(src.replace(orig, bad, 1), str(tmp_path / "mutant.so"))
    oracle.use(mutant)
    try:
        failed = failing_pins()
    finally:
        oracle.use(None)
    assert failed, f"no pin caught: {name}"


def test_real_oracle_passes_every_pin():
    oracle.use(None)
    assert failing_pins() == []
