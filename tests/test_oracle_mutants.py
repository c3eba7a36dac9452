"""The oracle's pins catch plausible mistakes: each mutant below is oracle.c
with one deliberate error planted (on the CPU); the pin suite must fail on
every one of them."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("sphere far root", "double t = (-b - sq) / a;", "double t = (-b + sq) / a;"),
    ("dropped u+v term", "if (v < 0.0 || u + v > 1.0) return 0;", "if (v < 0.0) return 0;"),
    ("cross sign", "return mk(a.y * b.z - a.z * b.y,", "return mk(a.z * b.y - a.y * b.z,"),
    ("ambient", "#define K_AMBIENT 0.1", "#define K_AMBIENT 0.2"),
    ("reflection weight", "col = add(col, scl(c2, refl));", "col = add(col, scl(c2, 1.0 - refl));"),
    ("no normal flip", "if (dot(n, r.d) > 0.0) n = scl(n, -1.0);", ""),
    ("eyes swapped", "v3 o = add(k->eye, scl(k->right, eye * 0.5 * k->sep));",
     "v3 o = add(k->eye, scl(k->right, -eye * 0.5 * k->sep));"),
    ("rows flipped", "double ny = (1.0 - 2.0 * (j + 0.5) / k->H) * k->tanh_y;",
     "double ny = (2.0 * (j + 0.5) / k->H - 1.0) * k->tanh_y;"),
    ("toe-in window", "v3 q = add(k->eye, scl(add(k->fwd, add(scl(k->right, nx), scl(k->up, ny))), k->zc));",
     "v3 q = add(k->eye, scl(add(k->fwd, add(scl(k->right, nx), scl(k->up, ny))), 0.5 * k->zc));"),
    ("morton axis", "m |= ((qx >> k) & 1u) << (3 * k + 2);", "m |= ((qx >> k) & 1u) << (3 * k + 1);"),
    ("quantisation scale", "double f = floor((c - lo) / ext * 1024.0);", "double f = floor((c - lo) / ext * 1023.0);"),
    ("split predicate", "if (clz64(s->keys[a] ^ s->keys[i]) > dn) gamma = i;",
     "if (clz64(s->keys[a] ^ s->keys[i]) >= dn) gamma = i;"),
    ("tie break", "if (t < best->t || (t == best->t && id < best->id))",
     "if (t < best->t || (t == best->t && id > best->id))"),
    ("depth off by one", "if (refl > 0.0 && depth < tc->max_depth) {", "if (refl > 0.0 && depth <= tc->max_depth) {"),
    ("box not outward", "if ((double)f < s || ((double)f == s && err > 0.0)) f = nextafterf(f, INFINITY);", ""),
    ("shadow ignored", "if (!occ) lsum += (double)s->li[l].intensity * ndl;", "lsum += (double)s->li[l].intensity * ndl;"),
    ("light vector sign", "v3 lv = sub(vf(s->li[l].pos), o2);", "v3 lv = sub(o2, vf(s->li[l].pos));"),
    ("no near tie at the shadow cut-off",
     "if (!is_best && fabs(t - tlim) * dl <= fmax(TIE_REL * tlim * dl, delta_k)) return 1;", ""),
    ("no near tie for a grazing light", "if (fabs(ndl) < TIE_REL) tc->flagged = 1;", ""),
]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, orig, bad, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site not unique: {orig}"
    mut = tmp_path / "oracle_mutant.c"
    mut.write_text(src.replace(orig, bad))
    lib = oracle.build(src=str(mut), out=str(tmp_path / "liboracle_mutant.so"))
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"the pins did not catch the mutant '{name}'"


# The network oracle (oracle/reproj.py) with one BF16 rounding point dropped
# or moved: the exact rounding-point pins must fail on each.
REPROJ_SRC = os.path.join(ROOT, "oracle", "reproj.py")
REPROJ_MUTANTS = [
    ("forward: weights unrounded", "            wt = _bf16(wt)\n", "            pass\n", "forward"),
    ("forward: hidden activations unrounded", "                x = _bf16(x)\n", "                pass\n",
     "forward"),
    ("forward: input unrounded", "        x = _bf16(x)\n    layers = unpack(params)",
     "        pass\n    layers = unpack(params)", "forward"),
    ("backward: input unrounded",
     "a = [rb(torch.tensor(np.asarray(feat, np.float64)[:, :IN_CH].reshape(H, W, IN_CH)).permute(2, 0, 1)[None])]",
     "a = [torch.tensor(np.asarray(feat, np.float64)[:, :IN_CH].reshape(H, W, IN_CH)).permute(2, 0, 1)[None]]",
     "grads"),
    ("backward: hidden activations unrounded",
     "a.append(rb(torch.relu(F.conv2d(a[-1], rb(w), b, padding=1))))",
     "a.append(torch.relu(F.conv2d(a[-1], rb(w), b, padding=1)))", "grads"),
    ("backward: data-gradient weights unrounded",
     "da = G.conv2d_input(a[li].shape, rb(w), dz_in, padding=1)",
     "da = G.conv2d_input(a[li].shape, w, dz_in, padding=1)", "grads"),
    ("backward: p - y rounded for the layer-4 weight gradient", "    dz = g\n", "    dz = rb(g)\n", "grads"),
    ("backward: p - y unrounded for the data gradient", "dz_in = rb(g)", "dz_in = g", "grads"),
    ("backward: masked data gradient unrounded", "dz = rb(da * (a[li] > 0))", "dz = da * (a[li] > 0)",
     "grads"),
]


@pytest.mark.parametrize("name,orig,bad,which", REPROJ_MUTANTS, ids=[m[0] for m in REPROJ_MUTANTS])
def test_network_pins_catch_planted_mistake(name, orig, bad, which):
    import types

    from tests import test_oracle_reproj as pins
    src = open(REPROJ_SRC).read()
    assert src.count(orig) == 1, f"mutation site not unique: {orig!r}"
    mod = types.ModuleType("reproj_mutant")
    exec(compile(src.replace(orig, bad), "reproj_mutant.py", "exec"), mod.__dict__)
    check = pins.check_forward_bf16 if which == "forward" else pins.check_grads_bf16
    with pytest.raises(AssertionError):
        check(mod)
