"""The FP64 oracle against its pins (CPU only).

Each pin of ``tests/pins.py`` runs as its own test.  ``test_planted_mistake``
then plants plausible mistakes in a temporary copy of the oracle source (a
dropped factor, a flipped sign, a transposed operand, an off-by-one), builds
it, and checks that the pin battery rejects every mutant.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests import pins

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin, orc):
    pin(orc)


# (original text, mutated text, what the mistake is)
MUTANTS = [
    ("double b = (double)deg * sqrt(dx * dx + dy * dy);",
     "double b = sqrt(dx * dx + dy * dy);", "B without the degree factor"),
    ("double lim = s->B * (b - a);", "double lim = s->B;", "sub-ellipse not scaled by b-a"),
    ("acc->ang += atan2(ax * by - ay * bx, ax * bx + ay * by);",
     "acc->ang += atan2(ay * bx - ax * by, ax * bx + ay * by);", "chord angle sign"),
    ("q[2 * i] = (1.0 - t) * q[2 * i] + t * q[2 * i + 2];",
     "q[2 * i] = t * q[2 * i] + (1.0 - t) * q[2 * i + 2];", "de Casteljau weights swapped"),
    ("return seg_wn(s, px, py, m, b, gm, gb, eps, depth + 1, acc);",
     "return seg_wn(s, px, py, m, b, ga, gb, eps, depth + 1, acc);", "wrong endpoint on recursion"),
    ("or_eval_w(s->deg, s->P, s->W, m, gm);", "or_eval_w(s->deg, s->P, s->W, 0.5, gm);", "midpoint of the root"),
    ("acc->half += cr > 0 ? 1 : -1;", "acc->half += cr > 0 ? -1 : 1;", "line-term side"),
    ("double klo = ceil(sp - L->smax), khi",
     "double klo = ceil(sp - L->smax) + 1.0, khi", "slab window off by one"),
    ("acc->ang -= chord_angle(qx, qy, L->g0, L->g0v);",
     "acc->ang += chord_angle(qx, qy, L->g0, L->g0v);", "chord correction sign"),
    ("long I = (Pu > 0) ? lround_d((ex - P[0]) / Pu) : 0;",
     "long I = (Pu > 0) ? lround_d((P[0] - ex) / Pu) : 0;", "lifting shift direction"),
    ("long I = (long)c * D->i0, J = (long)c * D->j0;\n                bnd",
     "long I = (long)c * D->j0, J = (long)c * D->i0;\n                bnd", "family generator transposed"),
    ("if (!(wb > 0)) continue;", "if (wb > 0) continue;", "farthest instead of nearest pair"),
    ("if (Pv > 0) L->hq = (int)lround_d((e->P[2 * e->deg + 1] - f->P[1]) / Pv);",
     "if (Pv > 0) L->hq = (int)lround_d((e->P[2 * e->deg] - f->P[0]) / Pv);", "homology axes mixed"),
    ("*state = (om >= 0.5) ? OR_INSIDE : OR_OUTSIDE;",
     "*state = (om > 0.0) ? OR_INSIDE : OR_OUTSIDE;", "classification threshold"),
    ("double clo = ceil((np - D->phi[k]) / PP), chi = floor((np - D->plo[k]) / PP);",
     "double clo = ceil((np - D->plo[k]) / PP), chi = floor((np - D->plo[k]) / PP);",
     "family window edge"),
    ("out[0] = h[0] / h[2];", "out[0] = h[0];", "rational point not divided by its weight"),
    ("h[3 * i + 2] = W[i];", "h[3 * i + 2] = 1.0;", "rational denominator without the weights"),
    ("const double b1 = (double)deg * r * dall, b2 = (double)deg * r * r * dnext;",
     "const double b1 = (double)deg * dall, b2 = (double)deg * dnext;", "rational bound without the weight ratio"),
    ("D->seg[s].W = D->w ? D->w + off : NULL;", "D->seg[s].W = D->w ? D->w : NULL;",
     "first segment's weights for every segment"),
    ("if (Pu > 0) copies_1d(x, L->box[0], L->box[1], Pu, &ia, &ib);",
     "if (Pv > 0) copies_1d(x, L->box[0], L->box[1], Pu, &ia, &ib);",
     "u-cylinder contractible copies gated on the v period (only the i = 0 copy)"),
    ("if (Pv > 0) copies_1d(y, L->box[2], L->box[3], Pv, &ja, &jb);",
     "if (Pv > 0 && Pu > 0) copies_1d(y, L->box[2], L->box[3], Pv, &ja, &jb);",
     "v-cylinder contractible copies skipped (only the j = 0 copy)"),
    ("if (!(xs >= L->box[0] && xs <= L->box[1])) continue;",
     "if (!(xs >= L->box[2] && xs <= L->box[3])) continue;",
     "contractible copy window on the wrong axis's range"),
]

# fast pins first, so that most mutants fail within a second
BATTERY = [pins.pin_single_chord, pins.pin_circles, pins.pin_polygon_exact,
           pins.pin_classification, pins.pin_hull_oracle, pins.pin_bound_contains_curve,
           pins.pin_eval, pins.pin_additivity_elevation_reversal, pins.pin_unit_jump,
           pins.pin_cylinder_closed_form, pins.pin_torus_bands, pins.pin_lift_homology,
           pins.pin_window_enlargement, pins.pin_lattice_translate, pins.pin_unfold_3x3,
           pins.pin_cylinder_unfold,
           pins.pin_config1_integers, pins.pin_rational_circle_arcs, pins.pin_rational_bound,
           pins.pin_rational_invariants, pins.pin_rational_dense_polyline]


def _build_mutant(src_text, tmpdir, idx):
    c = os.path.join(tmpdir, f"m{idx}.c")
    so = os.path.join(tmpdir, f"libm{idx}.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                    "-fPIC", "-shared", "-pthread", c, "-o", so, "-lm"], check=True)
    return so


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[2] for m in MUTANTS])
def test_planted_mistake(k, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "wn_oracle.c")).read()
    orig, mut, what = MUTANTS[k]
    assert src.count(orig) == 1, f"mutation anchor not found once: {what}"
    so = _build_mutant(src.replace(orig, mut), str(tmp_path), k)
    L = oracle.lib(so)
    caught = None
    for pin in BATTERY:
        try:
            with np.errstate(all="ignore"):
                pin(L)
        except (AssertionError, oracle.OracleError, ValueError, IndexError, OverflowError) as e:
            caught = pin.__name__
            break
    assert caught is not None, f"no pin caught the planted mistake: {what}"


def test_threads_agree(orc):
    """Splitting queries over threads does not change any result."""
    import wn_synth as ws
    dom, q = ws.config1(n_uniform=5000, n_near=500)
    w1, s1 = oracle.query(dom, q, threads=1, L=orc)
    w8, s8 = oracle.query(dom, q, threads=8, L=orc)
    assert np.array_equal(s1, s8)
    assert np.array_equal(w1, w8)
