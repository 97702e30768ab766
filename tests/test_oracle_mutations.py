"""The oracle's pins must catch plausible mistakes: each case compiles a copy
of the oracle with one planted error (a dropped factor, a wrong sign, index
or operand) on the CPU and checks that the pin tests fail on it."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gmr_oracle.cpp")
PINS = ["tests/test_oracle_convert.py", "tests/test_oracle_render.py", "tests/test_oracle_grad.py",
        "tests/test_oracle_sh.py"]

MUTATIONS = {
    "jacobian_z_sign": ("dt[2] += dJ[0] * (-fx / (z * z));", "dt[2] += dJ[0] * (fx / (z * z));"),
    "dM_factor": ("dM[3 * r + q] = 2.0 * (GS", "dM[3 * r + q] = 1.0 * (GS"),
    "conic_offdiag_half": ("{fg.dQ[0], 0.5 * fg.dQ[1]}", "{fg.dQ[0], 1.0 * fg.dQ[1]}"),
    "moment_coefficient": ("+ fp * gp * T(1.0 / 12.0)", "+ fp * gp * T(1.0 / 6.0)"),
    "kappa_constant": ("T kappa = area / (T(kPi) *", "T kappa = area / (T(3.0) *"),
    "gram_schmidt_sign": ("dxk += -dot(dw, g.xa);", "dxk += dot(dw, g.xa);"),
    "suffix_division": ("- S[ch] / (1.0 - cb.alpha)", "- S[ch]"),
    "conic_index": ("t.du[0] = dpower * (-(pr.Q[0] * cb.dx + pr.Q[1] * cb.dy));",
                    "t.du[0] = dpower * (-(pr.Q[0] * cb.dx + pr.Q[2] * cb.dy));"),
    "jacobian_operand": ("p.J[2] = -fx * x / (z * z);", "p.J[2] = -fx * y / (z * z);"),
    "add_after_stop": ("if (val(test) < kTMin) break;",
                       "if (val(test) < kTMin) { for (int ch = 0; ch < 3; ++ch) "
                       "C[ch] += P.col[3 * (size_t)f + ch] * alpha * Tr; Tr = test; break; }"),
    "eigen_swap": ("T sx2 = kappa * lam1, sy2 = kappa * lam2", "T sx2 = kappa * lam2, sy2 = kappa * lam1"),
    "centroid_component": ("V3<T> m = vi + mux * xa + muy * ya;", "V3<T> m = vi + mux * xa + mux * ya;"),
    "normal_cross_order": ("dya = dya + cross(dnv, g.xa);", "dya = dya + cross(g.xa, dnv);"),
    "rect_too_small": ("rx = rx + 0.25f;", "rx = rx - 1.5f;"),
    "sh_basis_component": ("Y[1] = T(kSh.c1) * y;", "Y[1] = T(kSh.c1) * x;"),
    "sh_tangent_projection": ("(1.0 / rn) * (dd - dot(d, dd) * d)", "(1.0 / rn) * (dd + dot(d, dd) * d)"),
    "sh_grad_factor": ("G[6][2] = kSh.c2b * 6.0 * z;", "G[6][2] = kSh.c2b * 3.0 * z;"),
    "depth_order": ("return bins[(size_t)view * F + i].depth_bits < bins[(size_t)view * F + j].depth_bits;",
                    "return bins[(size_t)view * F + i].depth_bits > bins[(size_t)view * F + j].depth_bits;"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(SRC).read()
    a, b = MUTATIONS[name]
    assert src.count(a) == 1, "mutation anchor must match exactly once"
    cpp = tmp_path / "mutant.cpp"
    lib = tmp_path / "libmutant.so"
    cpp.write_text(src.replace(a, b))
    sys.path.insert(0, ROOT)
    from oracle import build as obuild

    subprocess.run(["g++", *obuild.FLAGS, "-o", str(lib), str(cpp)], check=True)
    env = dict(os.environ, GMR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS, cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} was not caught:\n{r.stdout[-2000:]}"
    # caught by a failing pin, not by a mutant that does not load
    assert "OSError" not in r.stdout and "undefined symbol" not in r.stdout, r.stdout[-2000:]
    assert " passed" in r.stdout or "1 failed" in r.stdout, r.stdout[-2000:]
