"""Plant plausible mistakes in a copy of the CPU oracle and check that the
oracle's pins catch every one.

Each mutant is a text edit of one oracle source file (a wrong sign, a swapped
left/right index, a dropped factor, the limiter looking downwind, ...).  The
copy is compiled into a temporary directory and the pin suite runs against it
in a subprocess (through ORC_LIB); the pins must fail.  Nothing here touches a
GPU, and the real oracle sources are only read.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (file, original text, mutated text, what the slip is[, n]): the text must
# be unique in the file, or n picks its n-th occurrence (lines the Roe and
# the bathymetry solvers share)
MUTANTS = [
    ("orc_acoustics.c", "double alpha2 = (dp + Z_l * du) / (Z_l + Z_r);",
     "double alpha2 = (dp - Z_l * du) / (Z_l + Z_r);", "sign of a wave strength"),
    ("orc_acoustics.c", "W[0][0] = -alpha1 * Z_l;", "W[0][0] = -alpha1 * Z_r;",
     "left/right impedance swapped"),
    ("orc_acoustics.c", "s[0] = -c_l;", "s[0] = -c_r;", "left-going speed from the wrong cell"),
    ("orc_shallow_water.c", "double alpha2 = d2 - v_hat * d0;",
     "double alpha2 = d2 - u_hat * d0;", "shear strength uses the normal velocity"),
    ("orc_shallow_water.c",
     "double u_hat = (sqh_l * u_l + sqh_r * u_r) / (sqh_l + sqh_r);",
     "double u_hat = (sqh_r * u_l + sqh_l * u_r) / (sqh_l + sqh_r);", "Roe weights swapped", 1),
    ("orc_shallow_water.c", "double beta = (lam_m - s[0]) / (lam_m - lam_l);",
     "double beta = (s[0] - lam_l) / (lam_m - lam_l);", "entropy-fix fraction transposed"),
    ("orc_shallow_water.c", "if (lam_l < 0.0 && 0.0 < lam_m) {",
     "if (lam_l < 0.0 || 0.0 < lam_m) {", "entropy fix triggers off the sonic point"),
    ("orc_shallow_water.c", "double c_hat = sqrt(g * h_bar);",
     "double c_hat = sqrt(g * h_r);", "Roe celerity from one side", 1),
    ("orc_wavesweep.c", "int J = w->s[I + 1][p] > 0.0 ? I - 1 : I + 1;",
     "int J = w->s[I + 1][p] > 0.0 ? I + 1 : I - 1;", "limiter looks downwind"),
    ("orc_wavesweep.c", "if (dot_ii != 0.0) phi = orc_phi(P->limiter, dot_ji / dot_ii);",
     "if (dot_ji != 0.0) phi = orc_phi(P->limiter, dot_ii / dot_ji);", "theta ratio inverted"),
    ("orc_wavesweep.c", "acc += k * (1.0 - nu * as) * w->Wt[I + 1][p][c];",
     "acc += k * w->Wt[I + 1][p][c];", "dropped (1 - nu|s|) factor"),
    ("orc_wavesweep.c", "w->F[I + 1][c] = 0.5 * acc;", "w->F[I + 1][c] = acc;",
     "dropped 1/2 in the correction flux"),
    ("orc_wavesweep.c", "double first = w->apdq[i + 1][c] + w->amdq[i + 2][c];",
     "double first = w->apdq[i + 1][c] + w->amdq[i + 1][c];", "fluctuation from the wrong interface"),
    ("orc_wavesweep.c", "double second = w->F[i + 2][c] - w->F[i + 1][c];",
     "double second = w->F[i + 1][c] - w->F[i + 2][c];", "correction flux difference reversed"),
    ("orc_wavesweep.c", "    *sign = -1.0;\n", "    *sign = 1.0;\n", "wall does not reflect"),
    ("orc_wavesweep.c", "return lo ? i + N : i - N;", "return lo ? i + N : i - N + 1;",
     "periodic wrap off by one"),
    ("orc_wavesweep.c", "return lo ? 0 : N - 1;", "return lo ? 1 : N - 2;",
     "extrapolation from the second cell"),
    ("orc_wavesweep.c", "double a = 0.5 * (1.0 + theta);", "double a = (1.0 + theta);",
     "MC centred slope without the 1/2"),
    ("orc_wavesweep.c", "double dt = M > 0.0 ? P->cfl_desired / M : P->dt_max;",
     "double dt = M > 0.0 ? P->cfl_max / M : P->dt_max;", "next step at cfl_max"),
    ("orc_wavesweep.c", "for (int d = 0; d < P->ndim; ++d) { dirs[n] = d; frac[n] = 1.0; ++n; }",
     "for (int d = P->ndim - 1; d >= 0; --d) { dirs[n] = d; frac[n] = 1.0; ++n; }",
     "sweeps in y, x order"),
    ("orc_wavesweep.c", "    return 2 - d;", "    return 1 + d;", "transverse momentum mapped to the normal one"),
    ("orc_wavesweep.c", "for (int c = 0; c < nq; ++c) w->Wt[I + 1][p][c] = 0.0;",
     "for (int c = 0; c < nq; ++c) w->Wt[I + 1][p][c] = w->W[I + 1][p][c];",
     "first-order method keeps the unlimited correction"),
    ("orc_wavesweep.c", "dirs[n] = P->ndim - 1; frac[n] = 1.0; ++n;",
     "dirs[n] = P->ndim - 1; frac[n] = 0.5; ++n;", "Strang middle sweep takes half a step"),
    ("orc_shallow_water.c", "g * h_bar * ((h_r - h_l) + (B_r - B_l));",
     "g * h_bar * (h_r - h_l);", "bathymetry source dropped"),
    ("orc_shallow_water.c", "g * h_bar * ((h_r - h_l) + (B_r - B_l));",
     "g * h_bar * ((h_r - h_l) - (B_r - B_l));", "bathymetry source with the wrong sign"),
    ("orc_shallow_water.c", "g * h_bar * ((h_r - h_l) + (B_r - B_l));",
     "g * h_r * ((h_r - h_l) + (B_r - B_l));", "source depth from one side"),
    ("orc_wavesweep.c", "double k = fwave ? (sp > 0.0 ? 1.0 : (sp < 0.0 ? -1.0 : 0.0)) : as;",
     "double k = as;", "f-wave correction weighted by |s| instead of sign(s)"),
    ("orc_unsplit.c", "flux_t[3 * kb + c] -= 0.5 * nu[d] * fm[c];\n                        flux_t[3 * ka + c] -= 0.5 * nu[d] * fp[c];",
     "(void)fm; (void)fp;", "unsplit update without transverse terms"),
    ("orc_unsplit.c", "flux_t[3 * kb + c] -= 0.5 * nu[d] * fm[c];\n                        flux_t[3 * ka + c] -= 0.5 * nu[d] * fp[c];",
     "flux_t[3 * kb + c] += 0.5 * nu[d] * fm[c];\n                        flux_t[3 * ka + c] += 0.5 * nu[d] * fp[c];",
     "transverse terms with the wrong sign"),
    ("orc_unsplit.c", "double al = (-a[0] + Z_c * a[2]) / (Z_d + Z_c);",
     "double al = (-a[0] + Z_c * a[2]) / (Z_u + Z_c);", "transverse split with the wrong neighbour's impedance"),
    ("orc_unsplit.c", "double lam[3] = {vt - ct, vt, vt + ct};",
     "double lam[3] = {ut - ct, ut, ut + ct};", "transverse speeds from the velocity along the sweep"),
    ("orc_unsplit.c", "if (I - 1 >= 0) for (int c = 0; c < 3; ++c) fl[3 * (d * np + pidx(&u, il, jl)) + c] += fa[c];",
     "if (I - 1 >= 0) for (int c = 0; c < 3; ++c) fl[3 * (d * np + pidx(&u, il, jl)) + c] += fb[c];",
     "left fluctuation taken from the wrong side"),
    # wetting and drying (hydrostatic reconstruction around HLLE)
    ("orc_shallow_water.c", "double lam_rp = wet_r ? u_r + c_r : u_l + 2.0 * c_l;",
     "double lam_rp = wet_r ? u_r + c_r : u_l + c_l;", "dry-bed front at u + c instead of u + 2c"),
    ("orc_shallow_water.c", "double Bs = B_l > B_r ? B_l : B_r;",
     "double Bs = B_l < B_r ? B_l : B_r;", "reconstruction against the lower bed"),
    ("orc_shallow_water.c", "amdq[c] = (hl - h_l) * cut_l[c];", "amdq[c] = 0.0;",
     "momentum the reconstruction removes is lost"),
    ("orc_shallow_water.c", "double s1 = u_hat - c_hat < lam_lm ? u_hat - c_hat : lam_lm;",
     "double s1 = u_hat - c_hat;", "Roe speed instead of Einfeldt's"),
    ("orc_shallow_water.c", "    if (!wet_l || !wet_r)\n        for (int p = 0; p < 3; ++p)",
     "    if (0)\n        for (int p = 0; p < 3; ++p)", "correction kept at the shoreline"),
    ("orc_shallow_water.c", "W[2][c] = (df - s1 * dq) / (s3 - s1);",
     "W[2][c] = (df - s3 * dq) / (s3 - s1);", "HLL wave with the wrong speed"),
]


def _build_mutant(tmp, fname, old, new, nth=None):
    src_dir = os.path.join(tmp, "src")
    os.makedirs(src_dir, exist_ok=True)
    for f in os.listdir(ORACLE):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(ORACLE, f), src_dir)
    path = os.path.join(src_dir, fname)
    text = open(path).read()
    if nth is None:
        assert text.count(old) == 1, f"pattern not unique in {fname}: {old!r}"
        text = text.replace(old, new)
    else:
        assert text.count(old) >= nth, f"pattern occurs fewer than {nth} times in {fname}"
        at = -1
        for _ in range(nth):
            at = text.index(old, at + 1)
        text = text[:at] + new + text[at + len(old):]
    open(path, "w").write(text)
    lib = os.path.join(tmp, "libmut.so")
    cfiles = [os.path.join(src_dir, f) for f in sorted(os.listdir(src_dir)) if f.endswith(".c")]
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-fopenmp",
                    "-shared", "-o", lib] + cfiles + ["-lm"], check=True)
    return lib


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[3] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, mutant):
    fname, old, new, what = mutant[:4]
    lib = _build_mutant(str(tmp_path), fname, old, new, *mutant[4:])
    env = dict(os.environ, ORC_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_dry_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutant: {what}\n{r.stdout[-2000:]}"
