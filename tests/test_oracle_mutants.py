"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU, in a
temporary directory), builds it, swaps it in for the real oracle library and
runs the pin tests: at least one pin must fail for every mutant, and all of
them must pass for the unmodified source.
"""
import os
import shutil

import pytest

import oracle
from tests import test_oracle_pins as pins

PIN_CASES = [
    (pins.test_invariants_tiny, {}),
    (pins.test_walk_equals_bruteforce_tiny_camera, {}),
    (pins.test_walk_equals_bruteforce_random_meshes, {"seed": 11}),
    (pins.test_closed_form_plane, {"direction": 1}),
    (pins.test_closed_form_plane, {"direction": -1}),
    (pins.test_closed_form_sphere, {}),
    (pins.test_restart_rays_equal_bruteforce, {}),
    (pins.test_locate_contains_point, {}),
    (pins.test_asymmetry_checker_counts_planted_links, {}),
]

MUTANTS = {
    "face_winding": ("{{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}}",
                     "{{1, 2, 3}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}}"),
    "cross_dropped_term": ("r[2] = a[0] * b[1] - a[1] * b[0];", "r[2] = a[0] * b[1];"),
    "exit_sign": ("if (nd < 0.0) {", "if (nd > 0.0) {"),
    "mt_swapped_bary": ("*b1 = dot3(s, p) * inv;", "*b1 = dot3(d, q) * inv; (void)p;"),
    "tmax_ignored": ("if (tbest > tmax) break;", "(void)tmax;"),
    "side_flipped": ("m->ctet[2 * c + (s > 0 ? 0 : 1)] = t;", "m->ctet[2 * c + (s > 0 ? 1 : 0)] = t;"),
    "wrong_neighbour_face": ("kin = m->nbrk[4 * T + best];", "kin = best;"),
    # the builder writes a wrong back-link index for one side of every face
    "nbrk_backlink": ("m->nbrk[o1] = o0 % 4;", "m->nbrk[o1] = (o0 + 1) % 4;"),
    # the symmetry checker loses its back-link test, or its vertex comparison
    "asym_no_backlink_check": ("if (m->nbr[4 * u + ku] != t) { ++bad; continue; }",
                               "if (m->nbr[4 * u + ku] != t) { continue; }"),
    "asym_no_vertex_check": ("if (a != x || b != y || c != z) ++bad;", "(void)x; (void)y; (void)z;"),
}


def run_pins():
    failed = 0
    for fn, kw in PIN_CASES:
        try:
            fn(**kw)
        except Exception:  # any pin failure or error counts
            failed += 1
    return failed


def build_variant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    return oracle.load(oracle.build(str(path), str(tmp_path / f"lib{name}.so")))


def test_broken_backlink_is_reported_by_the_checker(tmp_path, monkeypatch):
    """With the builder's back-link broken, the symmetry checker itself (not
    only the walk pins) reports the broken links on a valid mesh."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    import scenegen as sg
    lib = build_variant(tmp_path, "nbrk_backlink", *MUTANTS["nbrk_backlink"])
    s = sg.make_config("tiny")
    m = oracle.OracleMesh(s.points, s.tets, s.tris, lib=lib)
    interior = 4 * s.n_tets - 12 * s.n * s.n
    assert m.count_asymmetric() >= interior // 2


def test_unmodified_oracle_passes_pins():
    assert run_pins() == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    lib = build_variant(tmp_path, name, *MUTANTS[name])
    monkeypatch.setattr(oracle, "_lib", lib)
    assert run_pins() > 0, f"no pin caught the planted mistake {name}"


# Mistakes planted in a copy of the secondary-ray generators (oracle/secondary.py),
# loaded as a separate module; the pins of tests/test_oracle_rays.py run on it.
GEN_MUTANTS = {
    "eta_inverted": ("eta = np.where(side == 1, float(ior), 1.0 / float(ior))",
                     "eta = np.where(side == 1, 1.0 / float(ior), float(ior))"),
    "mirror_sign": ("refl = w + (2.0 * cs)[:, None] * na", "refl = w - (2.0 * cs)[:, None] * na"),
    "refract_side": ("out_side = np.where(ok, 1 - side, side)", "out_side = side"),
    "shadow_side": ('side = np.where(np.einsum("ij,ij->i", nrm, L - v0) >= 0.0, 0, 1)',
                    'side = np.where(np.einsum("ij,ij->i", nrm, L - v0) >= 0.0, 1, 0)'),
    "snell_root_sign": ("(eta * cs - np.sqrt(np.maximum(k, 0.0)))",
                        "(eta * cs + np.sqrt(np.maximum(k, 0.0)))"),
    "normal_not_turned": ("na = np.where((side == 1)[:, None], -n, n)", "na = n"),
    "shadow_tmax_short": ("ln.astype(np.float32),", "(0.99 * ln).astype(np.float32),"),
}


def load_generators(name=None):
    import importlib.util
    import types
    from oracle import secondary
    src = open(secondary.__file__).read()
    if name is not None:
        old, new = GEN_MUTANTS[name]
        assert src.count(old) == 1, f"mutation site for {name} not unique"
        src = src.replace(old, new)
    mod = types.ModuleType(f"secondary_{name}")
    exec(compile(src, f"<secondary {name}>", "exec"), mod.__dict__)
    return mod


def run_generator_pins(mod):
    from tests import test_oracle_rays as rays
    failed = 0
    for check in rays.CHECKS:
        try:
            check(mod)
        except Exception:
            failed += 1
    return failed


def test_unmodified_generators_pass_pins():
    assert run_generator_pins(load_generators()) == 0


@pytest.mark.parametrize("name", sorted(GEN_MUTANTS))
def test_generator_mutant_is_caught(name):
    assert run_generator_pins(load_generators(name)) > 0, f"no pin caught {name}"
