"""The oracle's pins catch plausible mistakes in the oracle itself.

Each case below plants one mistake in a copy of ``oracle/oracle.c`` (a
dropped term, a transposed or unconjugated operand, a wrong sign, index or
normalisation), compiles the copy into a temporary library, points the oracle
wrapper at it and runs every pin of ``test_oracle_pins.py``.  At least one pin
that does not rest on the oracle's own stored output (most often several)
must fail: the fixtures under ``tests/golden/`` were written by the oracle and
only guard against regressions, so they are not counted.  The oracle source
on disk is never changed.
"""
import inspect
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text in oracle.c, replacement, least number of independent pins that must fail)
MUTANTS = [
    # Eq. (def_hamilton): the B'^H (T^BA A + T^BB B) half of the sum left out
    ("h_drops_b_rows", "h += ca * ya[L] + cb * ya[nl + L];", "h += ca * ya[L];", 4),
    # Eq. (def_overlap): the A^H A term left out
    ("s_drops_a_term", "sa[L] = w[L];", "sa[L] = 0;", 4),
    # Eq. (def_overlap): the ||udot||^2 weight of the B^H B term left out
    ("s_drops_u2", "sa[nl + L] = u2 * w[nl + L];", "sa[nl + L] = w[nl + L];", 3),
    # U instead of U^2 (the reading of Eq. (s) with U^H U)
    ("s_uses_u_not_u2", "double u2 = U[t * (lmax + 1) + l] * U[t * (lmax + 1) + l];",
     "double u2 = U[t * (lmax + 1) + l];", 3),
    # T applied transposed (T^T = conj(T) for Hermitian T)
    ("h_transposed_t", "acc += Ta[(size_t)i * n2 + j] * w[j];",
     "acc += Ta[(size_t)j * n2 + i] * w[j];", 3),
    # the row operand not conjugated
    ("rows_not_conjugated", "double _Complex ca = conj((double _Complex)A[(size_t)a * nl + L]);",
     "double _Complex ca = (double _Complex)A[(size_t)a * nl + L];", 5),
    # 4 pi / Omega instead of 4 pi / sqrt(Omega)
    ("normalisation_omega", "real_t pref = 4 * PI_L / sqrtl(c->volume);",
     "real_t pref = 4 * PI_L / c->volume;", 4),
    # (-i)^l instead of i^l in the Rayleigh expansion
    ("i_power_sign", "(l % 4 == 1) ? I : (l % 4 == 2) ? -1 : -I;",
     "(l % 4 == 1) ? -I : (l % 4 == 2) ? -1 : I;", 3),
    # Y_lm(K_hat) instead of conj(Y_lm(K_hat))
    ("ylm_not_conjugated", "cplx_t f = pref * phase * il * conjl(Y[L]);",
     "cplx_t f = pref * phase * il * Y[L];", 3),
    # exp(-i K.tau) instead of exp(+i K.tau)
    ("phase_sign", "cplx_t phase = cosl(2 * PI_L * arg) + I * sinl(2 * PI_L * arg);",
     "cplx_t phase = cosl(2 * PI_L * arg) - I * sinl(2 * PI_L * arg);", 5),
    # a sign slip in Cramer's rule for B
    ("cramer_b_sign", "bl[t * (c->lmax + 1) + l] = (u * dj - up * j) / D;",
     "bl[t * (c->lmax + 1) + l] = (up * j - u * dj) / D;", 4),
    # j_l' = j_{l-1} - l/x j_l (should be (l+1)/x)
    ("bessel_derivative_index", "return jl(l - 1, x) - (l + 1) / x * jl(l, x);",
     "return jl(l - 1, x) - l / x * jl(l, x);", 7),
    # j_l for x >= l + 1: alternating signs of the sine polynomial lost
    ("bessel_trig_sign", "P += (k % 2 ? -c : c);", "P += c;", 6),
    # j_l for small x: (2l+2n-1) for (2l+2n+1) in the series denominator
    ("bessel_series_denominator", "term *= h / ((real_t)n * (real_t)(2 * l + 2 * n + 1));",
     "term *= h / ((real_t)n * (real_t)(2 * l + 2 * n - 1));", 9),
    # Legendre three-term recurrence with (l+m) for (l+m-1)
    ("legendre_recurrence_index", "- (l + m - 1) * plm2) / (l - m);", "- (l + m) * plm2) / (l - m);", 7),
    # Y_lm normalisation with (l+m)!/(l-m)! inverted
    ("ylm_factorial_ratio", "factl(l - m) / factl(l + m));", "factl(l + m) / factl(l - m));", 8),
    # Y_{l,-m} = conj(Y_lm) without the (-1)^m
    ("ylm_negative_m_sign", "Y[l * l + l - m] = ((m % 2) ? -1 : 1) * conjl(y);",
     "Y[l * l + l - m] = conjl(y);", 3),
    # K = q . rec read with the reciprocal lattice transposed (skewed cells)
    ("reciprocal_transposed",
     "for (int j = 0; j < 3; ++j) K[j] = q[0] * c->rec[j] + q[1] * c->rec[3 + j] + q[2] * c->rec[6 + j];",
     "for (int j = 0; j < 3; ++j) K[j] = q[0] * c->rec[3 * j] + q[1] * c->rec[3 * j + 1] + q[2] * c->rec[3 * j + 2];",
     3),
    # plane waves: the k-point shift left out of |k+G| <= K_max
    ("gvectors_drop_k", "double q1 = n1 + k[0], q2 = n2 + k[1], q3 = n3i + k[2];",
     "double q1 = n1, q2 = n2, q3 = n3i;", 1),
    # plane waves sorted by descending |k+G|
    ("gvectors_descending", "if (a->key != b->key) return a->key < b->key ? -1 : 1;",
     "if (a->key != b->key) return a->key < b->key ? 1 : -1;", 1),
    # plane waves: the search box too small to hold the whole ball
    ("gvectors_box_too_small", "6.283185307179586) + 2;", "6.283185307179586) - 2;", 1),
]


def pin_calls():
    """Every pin of test_oracle_pins.py as (name, zero-argument call)."""
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        if name == "test_bessel_vs_scipy":
            out += [(f"{name}[{l}]", (lambda l=l, fn=fn: fn(l))) for l in (0, 1, 4, 12)]
        else:
            assert not inspect.signature(fn).parameters, name
            out.append((name, fn))
    return out


def failing_pins():
    failed = []
    for name, call in pin_calls():
        try:
            call()
        except Exception:  # an assertion, or a numerical routine rejecting the output
            failed.append(name)
    return failed


def compile_variant(text, path):
    c_path = str(path) + ".c"
    with open(c_path, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(path), c_path, "-lm"], check=True)
    return str(path)


@pytest.fixture
def use_library(monkeypatch):
    def use(so_path):
        monkeypatch.setattr(oracle, "build", lambda force=False: so_path)
        monkeypatch.setattr(oracle, "_lib", None)
    return use


def test_unchanged_copy_passes_every_pin(tmp_path, use_library):
    """The harness itself: the oracle recompiled from an unchanged copy fails nothing."""
    with open(SRC) as f:
        src = f.read()
    use_library(compile_variant(src, tmp_path / "liboracle_copy.so"))
    assert failing_pins() == []


@pytest.mark.parametrize("name,old,new,least", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_pins(tmp_path, use_library, name, old, new, least):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"{name}: the text to change is not unique in oracle.c"
    use_library(compile_variant(src.replace(old, new), tmp_path / f"liboracle_{name}.so"))
    failed = [f for f in failing_pins() if not f.startswith("test_golden")]
    assert len(failed) >= least, (name, failed)
