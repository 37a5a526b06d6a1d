"""The C ABI library loads and exports every function include/claw.h declares,
the Python binding covers them, and argument validation rejects bad input
before any device call (these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_1805_08846_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(claw_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["claw_create", "claw_set_q", "claw_step", "claw_advance", "claw_max_speed",
                     "claw_get_q", "claw_run_steps", "claw_ensemble_create",
                     "claw_ensemble_run_steps", "claw_destroy", "claw_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(L.lib()._name)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(L._SIGS)


def _create(**over):
    args = dict(n=(8, 8), dx=(0.1, 0.1), m=3, mwaves=3, system="shallow_water",
                limiter="minmod", bc="extrap", params=L.make_params(precision=64))
    args.update(over)
    return L.claw_create(**args)


@pytest.mark.parametrize("over,needle", [
    (dict(m=4), "(m, mwaves)"),
    (dict(mwaves=2), "(m, mwaves)"),
    (dict(n=(1, 8)), "at least 2 cells"),
    (dict(n=(8, 0)), "at least 2 cells"),
    (dict(dx=(0.0, 0.1)), "dx[0]"),
    (dict(n=(8, 8, 8), dx=(0.1, 0.1, 0.1), m=3, mwaves=3), "2D only"),
    (dict(params=L.make_params(precision=16)), "precision"),
    (dict(params=L.make_params(cfl_desired=0.0)), "cfl_desired"),
    (dict(params=L.make_params(g=-1.0)), "g must be"),
    (dict(params=L.make_params(splitting=7)), "unknown splitting"),
    (dict(n=(8, 8, 8), dx=(0.1, 0.1, 0.1), system="acoustics", m=4, mwaves=2,
          params=L.make_params(splitting="unsplit")), "unsplit update covers"),
    (dict(system="shallow_water_bathy", params=L.make_params(splitting="unsplit")), "unsplit update covers"),
    (dict(system="shallow_water_dry", params=L.make_params(splitting="unsplit")), "unsplit update covers"),
    (dict(system="shallow_water_dry", params=L.make_params(dry_tol=-1.0)), "dry_tol"),
    (dict(system="acoustics", m=3, mwaves=2, params=L.make_params(rho=0.0)), "rho and K"),
    (dict(system=7), "unknown system"),
    (dict(limiter=9), "unknown limiter"),
    (dict(bc=[5, 1, 1, 1]), "unknown bc"),
])
def test_invalid_arguments_are_rejected_before_any_device_work(over, needle):
    with pytest.raises(L.ClawError) as ei:
        _create(**over)
    assert ei.value.status == L.CLAW_EINVAL
    assert needle in str(ei.value)


def test_ensemble_rejects_empty_and_mixed_dimensions():
    with pytest.raises(L.ClawError) as ei:
        L.claw_ensemble_create([], "shallow_water", "minmod", "periodic", L.make_params())
    assert ei.value.status == L.CLAW_EINVAL
    with pytest.raises(L.ClawError) as ei:
        L.claw_ensemble_create([((8, 8), (0.1, 0.1)), ((8, 8, 8), (0.1,) * 3)], "acoustics", "mc",
                               "wall", L.make_params())
    assert ei.value.status == L.CLAW_EINVAL


def test_null_solver_is_rejected():
    lib = L.lib()
    assert lib.claw_run_steps(None, 1) == L.CLAW_EINVAL
    assert lib.claw_step(None, 0.0, None) == L.CLAW_EINVAL
    assert lib.claw_run_fixed_steps(None, 2, 0.1, None) == L.CLAW_EINVAL
    assert lib.claw_get_rows(None, 0, 1, None, 0) == L.CLAW_EINVAL
    assert lib.claw_set_rows(None, 0, 1, None, 0) == L.CLAW_EINVAL
    assert lib.claw_checkpoint(None) == L.CLAW_EINVAL
    assert lib.claw_rollback(None) == L.CLAW_EINVAL
    lib.claw_destroy(None)


def declaration_comments():
    """{function: the comment block that precedes its declaration} -- the
    last comment before it, possibly across the other declarations of its
    group."""
    out = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        for m in re.finditer(r"^[a-z_ ]+\*?\s*\b(claw_[a-z0-9_]+)\s*\(", text, flags=re.M):
            before = text[:m.start()]
            end = before.rfind("*/")
            start = before.rfind("/*", 0, end)
            c = before[start:end] if end >= 0 else ""
            out[m.group(1)] = re.sub(r"\s+", " ", re.sub(r"\n\s*\*", " ", c))
    return out


def test_every_declared_call_cites_the_paper_or_says_it_has_no_counterpart():
    """Each exported call's comment names the passage of the paper that
    defines its operation (a section or an equation), or states that the
    paper has no counterpart."""
    comments = declaration_comments()
    assert set(comments) == set(declared_functions())
    missing = [n for n, c in comments.items()
               if not re.search(r"\b(Sec\.|Eq\.|Table)|no counterpart", c)]
    assert not missing, missing
