"""The pins must be able to fail: plant a plausible mistake in a copy of the oracle
(on the CPU), rebuild it, and check that at least one pin rejects it."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "echo_oracle.c")

PW = "tests/test_oracle_pointwise.py"
SC = "tests/test_oracle_scheme.py"

# (name, text in the oracle, replacement, pins expected to catch it)
MUTATIONS = [
    ("mp5 finite-volume weights",
     "(3.0 * um2 - 20.0 * um1 + 90.0 * u0 + 60.0 * up1 - 5.0 * up2) / 128.0",
     "(2.0 * um2 - 13.0 * um1 + 47.0 * u0 + 27.0 * up1 - 3.0 * up2) / 60.0",
     [PW + "::test_mp5_exact_on_quartics_when_smooth",
      SC + "::test_convergence_order_one_period"]),
    ("mp5 right state not mirrored",
     "double m[5] = {s6[5], s6[4], s6[3], s6[2], s6[1]};",
     "double m[5] = {s6[1], s6[2], s6[3], s6[4], s6[5]};",
     [SC + "::test_rhs_converges_to_exact_time_derivative"]),
    ("der fourth-difference coefficient",
     "+ 3.0 * d4 / 640.0", "+ 3.0 * d4 / 64.0",
     [PW + "::test_der_exact_on_polynomials"]),
    ("int high-order weights",
     "(-s[0] + 9.0 * s[1] + 9.0 * s[2] - s[3]) / 16.0",
     "(-s[0] + 8.0 * s[1] + 8.0 * s[2] - s[3]) / 14.0",
     [PW + "::test_int_exact_on_polynomials"]),
    ("induction flux sign",
     "f[5 + i] = v[d] * B[i] - v[i] * B[d];", "f[5 + i] = v[i] * B[d] - v[d] * B[i];",
     [PW + "::test_traveling_wave_identity"]),
    ("momentum flux drops E E",
     "w * v[i] * v[d] - E[i] * E[d] - B[i] * B[d]", "w * v[i] * v[d] - B[i] * B[d]",
     [PW + "::test_momentum_flux_trace"]),
    ("c2p residual drops (S.B)^2 term",
     "- q->SB * q->SB / (2.0 * W * W) - q->U;", "- q->U;",
     [PW + "::test_c2p_residual_vanishes_at_true_W"]),
    ("c2p derivative sign",
     "*df = 1.0 - dp + 0.5 * q->B2 * dv2", "*df = 1.0 + dp + 0.5 * q->B2 * dv2",
     [PW + "::test_c2p_derivative_matches_finite_difference"]),
    ("hll speed weights swapped",
     "fhat[c] = (ap * fL[c] + am * fR[c]", "fhat[c] = (am * fL[c] + ap * fR[c]",
     [PW + "::test_hll_upwind_when_supersonic"]),
    ("uct b-side jump sign",
     "return e4 + da - db;", "return e4 + da + db;",
     [PW + "::test_uct_reduces_to_hll_along_b"]),
    ("uct a/b speed weights swapped",
     "double wa[2] = {apa, ama}, wb[2] = {apb, amb};",
     "double wa[2] = {ama, apa}, wb[2] = {apb, amb};",
     [PW + "::test_uct_reduces_to_hll_without_transverse_variation"]),
    ("sweep stencil off by one",
     "s6[m] = prim[v * n + at(g, i, j, k, d, m - 2)];",
     "s6[m] = prim[v * n + at(g, i, j, k, d, m - 1)];",
     [SC + "::test_brute_force_rhs", SC + "::test_rhs_converges_to_exact_time_derivative"]),
    ("curl sign",
     "curl_edges(g, E, -1.0, rhs_b);", "curl_edges(g, E, 1.0, rhs_b);",
     [SC + "::test_rhs_converges_to_exact_time_derivative"]),
    ("edge speeds taken at the wrong neighbour",
     "long ea1 = at(g, i, j, k, b, 1);", "long ea1 = at(g, i, j, k, a, 1);",
     [SC + "::test_brute_force_rhs"]),
    ("mc slope limiter central term",
     "b = 0.5 * (up1 - um1)", "b = 1.0 * (up1 - um1)",
     [PW + "::test_linear_reconstruction_exact_on_lines_and_bounded"]),
    ("rk2 final weight",
     "cons[q] = 0.5 * u0[q] + 0.5 * (cons[q] + dt * rc[q]);",
     "cons[q] = 0.4 * u0[q] + 0.6 * (cons[q] + dt * rc[q]);",
     [SC + "::test_fast_variant_second_order"]),
    ("rk3 second-stage weight",
     "cons[q] = 0.75 * u0[q] + 0.25 * (cons[q] + dt * rc[q]);",
     "cons[q] = 0.7 * u0[q] + 0.3 * (cons[q] + dt * rc[q]);",
     [SC + "::test_convergence_order_one_period"]),
]


def _build(src_text, tmpdir):
    c = os.path.join(tmpdir, "mut.c")
    so = os.path.join(tmpdir, "libmut.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", c,
                    "-o", so, "-lm"], check=True, capture_output=True)
    return so


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_reject_mutation(name, old, new, pins):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    with tempfile.TemporaryDirectory() as tmp:
        so = _build(src.replace(old, new), tmp)
        env = dict(os.environ, ECHO_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"]
                           + pins, cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 1, "no pin caught '%s':\n%s" % (name, r.stdout[-2000:])
