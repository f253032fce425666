"""Planted mistakes: the oracle's pins must catch each of them.  Every mutant below is a copy of the FP64
oracle (ccs_oracle.c) with one plausible mistake in one step of the method: a wrong Bernstein basis or
derivative, a sign or corner in the crop of Algorithm 1, a transposed de Casteljau split, the other
weight convention of the Gregory patch (Sec. 3.2), wrong corners or a dropped term in the bounds of
Algorithm 2, a missing slab swap, a transposed leaf cell, the other split axis order, pruning on the exit
distance, the tie rules of the leaf key, a non-orthonormal local frame (Sec. 3.4), the screen-space
threshold (Sec. 3.3) and the centre of a coarser leaf, the box extension and the ray's transform
(Sec. 3.4), a dropped BVH child, and each part of the FP32 error model that flags rays for the parity
tests (a flag never set, boxes not inflated or deflated, neighbouring cells taken as far apart).  Each copy is compiled on the CPU and the quick pin files are
run against it (CCS_ORACLE_LIB); every run must fail, while the unchanged source passes the same way.
Mutants that cannot change an answer (the order in which children are visited, the 0/0 reading of a
weight whose Bernstein factor vanishes) are left out: the pins are right to let them through."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ccs_oracle.c")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_local.py", "tests/test_oracle_screen.py",
             "tests/test_oracle_shadow.py", "tests/test_oracle_flags.py", "tests/test_oracle_scene.py"]
SLOW = "tests/test_oracle_scene.py::test_agrees_with_dense_tessellation"

# (name, text in ccs_oracle.c (exactly once), replacement)
MUTANTS = [
    ("bernstein basis B1", "    B[1] = 3.0 * t * s * s;", "    B[1] = 3.0 * t * t * s;"),
    ("bernstein derivative sign", "    D[0] = -3.0 * s * s;", "    D[0] = 3.0 * s * s;"),
    ("crop twist sign", "    Q(1, 1) = add(add(Q(1, 0)", "    Q(1, 1) = sub(add(Q(1, 0)"),
    ("crop boundary corner", "Q(2, 0) = sub(Q(3, 0), scl(evalBezierDu(p, u1, v0), Du));",
     "Q(2, 0) = sub(Q(3, 0), scl(evalBezierDu(p, u0, v0), Du));"),
    ("split axis transposed", "idx[k] = axis == 0 ? 4 * r + k : 4 * k + r;",
     "idx[k] = axis == 0 ? 4 * k + r : 4 * r + k;"),
    ("split right half order", "R[idx[1]] = m123; R[idx[2]] = m23;", "R[idx[1]] = m23; R[idx[2]] = m123;"),
    ("gregory weight convention", "    case 0: return ratio_or_half(u, v);", "    case 0: return ratio_or_half(v, u);"),
    ("gregory bound corners", "hA[0] = gregory_h(0, u0, v1); hB[0] = gregory_h(0, u1, v0);",
     "hA[0] = gregory_h(0, u0, v0); hB[0] = gregory_h(0, u1, v1);"),
    ("bernstein maximum w1", "            w[a][0] = 3.0 * w1 * (1.0 - w1) * (1.0 - w1);",
     "            w[a][0] = 3.0 * w1 * w1 * (1.0 - w1);"),
    ("bernstein clamp w2", "(t1 < 2.0 / 3.0 ? t1 : t0)", "(t1 < 2.0 / 3.0 ? t0 : t1)"),
    ("displacement term dropped", "        for (int k = 0; k < 4; ++k) {\n            double wk",
     "        for (int k = 0; k < 3; ++k) {\n            double wk"),
    ("displacement weight transposed", "double wk = w[0][k & 1] * w[1][k >> 1];",
     "double wk = w[0][k >> 1] * w[1][k & 1];"),
    ("lower patch from the upper points", "        for (int k = 0; k < 4; ++k) p[INNER_SLOT[k]] = lo[k];",
     "        for (int k = 0; k < 4; ++k) p[INNER_SLOT[k]] = hi[k];"),
    ("slab swap missing", "        if (ta > tb) { double t = ta; ta = tb; tb = t; }\n", ""),
    ("leaf cell transposed", "    return (cv << L) | cu;", "    return (cu << L) | cv;"),
    ("split along v first",
     "    int su = (level + 1) / 2, sv = level / 2;\n    uint64_t szu",
     "    int su = level / 2, sv = (level + 1) / 2;\n    uint64_t szu"),
    ("prune on exit distance", "        if (N.t0 > lim) continue;", "        if (N.t1 > lim) continue;"),
    ("patch tie rule reversed", "    if (pid != b->pid) return pid < b->pid;", "    if (pid != b->pid) return pid > b->pid;"),
    ("cell tie rule reversed", "    return cell < b->cell;", "    return cell > b->cell;"),
    ("gregory displacement not added",
     "            hi = add(hi, d);\n            extend_box(&lo, &hi, tau);\n            diag[s]",
     "            extend_box(&lo, &hi, tau);\n            diag[s]"),
    ("gregory domain transposed",
     "calcPointsAndD(P->gl, 1, u0, u1, v0, v1, q, &d, NULL, NULL);\n            if (st) st->expand_greg++;",
     "calcPointsAndD(P->gl, 1, v0, v1, u0, u1, q, &d, NULL, NULL);\n            if (st) st->expand_greg++;"),
    ("local frame not orthogonalised", "    v3 x = sub(e, scl(z, dot3(e, z)));", "    v3 x = e;"),
    ("screen-space threshold", "diag < 0.5 * spread * t_entry;", "diag < spread * t_entry;"),
    ("bvh child dropped", "        stack[sp++] = nd->right;\n", ""),
    ("bezier evaluation transposed", "r = add(r, scl(p[4 * j + i], Bu[i] * Bv[j]));",
     "r = add(r, scl(p[4 * i + j], Bu[i] * Bv[j]));"),
    ("crop step size", "    double Du = (u1 - u0) / 3.0;", "    double Du = (u1 - u0) / 2.0;"),
    ("gregory inner slots transposed", "static const int INNER_SLOT[4] = {5, 6, 9, 10};",
     "static const int INNER_SLOT[4] = {5, 9, 6, 10};"),
    ("gregory blend base", "p[INNER_SLOT[k]] = add(pv, scl(sub(pu, pv), gregory_h(k, u, v)));",
     "p[INNER_SLOT[k]] = add(pu, scl(sub(pu, pv), gregory_h(k, u, v)));"),
    ("slab containment for a zero direction", "            if (o < l || o > h) return 0;",
     "            if (o < l && o > h) return 0;"),
    ("box extension doubled", "const double e = 0.5 * (tau - w);", "const double e = (tau - w);"),
    ("box extension scale", "return ldexp(1.0, -19) * (1.0 + oc.x + oc.y + oc.z);",
     "return ldexp(1.0, -18) * (1.0 + oc.x + oc.y + oc.z);"),
    ("ray direction not rotated", "l.d = rotate(P->R, r->d); }", "l.d = r->d; }"),
    ("flag: another patch never reported", "            flags |= 1;\n", ""),
    ("flag: far cell never reported", "            flags |= 2;\n", ""),
    ("flag: near misses not reported", "        if (l.n) flags |= 4;\n", ""),
    ("flag: hits without a strict leaf not reported", "    if (R > B) {", "    if (0) {"),
    ("flag: loose boxes not inflated",
     "        *lo = sub(*lo, v3make(eps, eps, eps));\n        *hi = add(*hi, v3make(eps, eps, eps));\n", ""),
    ("flag: strict boxes not deflated", "if (h[k] - l[k] > 2.0 * eps) { l[k] += eps; h[k] -= eps; }",
     "if (h[k] - l[k] > 2.0 * eps) { }"),
    ("flag: early loose leaves not reported", "        if (e->tl < b->t - fabs(b->t) * rel_t) flags |= 8;\n", ""),
    ("flag: neighbouring cells taken as far", "return du < -1 || du > 1 || dv < -1 || dv > 1;",
     "return du != 0 || dv != 0;"),
    ("screen leaf centre axis", "J->u_out[i] = (float)((double)(b.cell & ((1ull << J->L) - 1)) / cells + ldexp(0.5, -su));",
     "J->u_out[i] = (float)((double)(b.cell & ((1ull << J->L) - 1)) / cells + ldexp(0.5, -sv));"),
]


def _compile(src_text: str, out: str) -> None:
    c = out[:-3] + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, c,
                           "-lm", "-lpthread"])


def _pins_pass(lib: str) -> tuple:
    """Run the quick pin files against the oracle build `lib`; (passed, last lines of the output)."""
    env = dict(os.environ, CCS_ORACLE_LIB=lib, PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
           "--deselect", SLOW] + PIN_FILES
    try:
        p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return False, "timed out"
    return p.returncode == 0, (p.stdout + p.stderr).strip().splitlines()[-1:]


def _run(args):
    name, find, repl, src, tmp = args
    out = os.path.join(tmp, "m%02d.so" % MUTANTS.index((name, find, repl)) if find else "control.so")
    _compile(src if not find else src.replace(find, repl), out)
    return name, _pins_pass(out)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    for name, find, _ in MUTANTS:
        assert src.count(find) == 1, f"mutant site of '{name}' is not unique in ccs_oracle.c"
    jobs = [("control", None, None, src, str(tmp_path))] + [(n, f, r, src, str(tmp_path)) for n, f, r in MUTANTS]
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        results = dict(ex.map(_run, jobs))
    ok, tail = results.pop("control")
    assert ok, f"the unchanged oracle fails its pins under the mutant harness: {tail}"
    survivors = [n for n, (passed, _) in results.items() if passed]
    assert not survivors, f"planted mistakes that no pin catches: {survivors}"


# Planted mistakes in the network oracle (oracle/mlp.py): each is a list of (text, replacement) applied
# together, so that a mistake made consistently in the forward and the backward pass is covered too.
MLP_MUTANTS = [
    ("second ReLU dropped", [("    h2 = np.maximum(z2, 0.0)\n", "    h2 = z2\n"),
                             ("    dz2 = dh2 * (z2 > 0)\n", "    dz2 = dh2\n")]),
    ("first ReLU dropped", [("    h1 = np.maximum(z1, 0.0)\n", "    h1 = z1\n"),
                            ("    dz1 = dh1 * (z1 > 0)\n", "    dz1 = dh1\n")]),
    ("second layer transposed", [("    z2 = h1 @ W2.T + b2\n", "    z2 = h1 @ W2 + b2\n"),
                                 ("    dW2 = dz2.T @ h1\n", "    dW2 = (dz2.T @ h1).T\n"),
                                 ("    dh1 = dz2 @ W2\n", "    dh1 = dz2 @ W2.T\n")]),
    ("column-major parameters", [("        out.append(theta[k:k + n].reshape(s))\n",
                                  "        out.append(theta[k:k + n].reshape(s[::-1]).T)\n"),
                                 ("dtype=np.float64).reshape(-1) for p in parts])",
                                  "dtype=np.float64).T.reshape(-1) for p in parts])")]),
    ("cross-entropy gradient sign", [("    dz3[np.arange(B), y] -= 1.0\n", "    dz3[np.arange(B), y] += 1.0\n")]),
    ("batch mean dropped from the gradient", [("    dz3 /= B\n", "")]),
    ("bias gradient", [("    db2 = dz2.sum(0)\n", "    db2 = dz2.mean(0)\n")]),
    ("bf16 ties away from even", [("(u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16", "(u + 0x8000) >> 16 << 16")]),
    ("bf16 forward: second ReLU dropped", [("    h2 = bf16(np.maximum(z2, 0.0)).astype(np.float64)\n",
                                            "    h2 = bf16(z2).astype(np.float64)\n")]),
    ("bf16 forward: second layer transposed", [("    z2 = h1 @ bf16(W2).astype(np.float64).T + b2",
                                                "    z2 = h1 @ bf16(W2).astype(np.float64) + b2")]),
    ("bf16 forward: first bias dropped", [(".T + b1.astype(np.float32)\n", ".T\n")]),
]


def _py_pins_pass(test_file: str, bindings: dict) -> bool:
    """Run every test of tests/<test_file> with the given module attributes rebound (a fresh copy of the
    test module, so its seeded generators start over)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_pins_" + test_file[:-3], os.path.join(ROOT, "tests", test_file))
    pins = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(pins)
    for k, v in bindings.items():
        if hasattr(pins, k):
            setattr(pins, k, v)
    for name in sorted(n for n in dir(pins) if n.startswith("test_")):
        try:
            getattr(pins, name)()
        except Exception:
            return False
    return True


def _py_module(src_text: str, package: str = None):
    import types
    m = types.ModuleType("_mutant")
    if package:   # a module of the oracle package (relative imports resolve against it)
        m.__package__ = package
        m.__name__ = package + "._mutant"
    exec(compile(src_text, "mutant.py", "exec"), m.__dict__)
    return m


def _survivors(src: str, mutants, passes) -> list:
    survivors = []
    for name, edits in mutants:
        m = src
        for find, repl in edits:
            assert m.count(find) == 1, f"mutant site of '{name}' is not unique: {find!r}"
            m = m.replace(find, repl)
        if passes(m):
            survivors.append(name)
    return survivors


def test_every_planted_mistake_in_the_network_oracle_fails_a_pin():
    src = open(os.path.join(ROOT, "oracle", "mlp.py")).read()
    passes = lambda text: _py_pins_pass("test_oracle_mlp.py", {"mlp": _py_module(text)})
    assert passes(src), "the unchanged network oracle fails its pins in the harness"
    survivors = _survivors(src, MLP_MUTANTS, passes)
    assert not survivors, f"planted mistakes in the network oracle that no pin catches: {survivors}"


# Planted mistakes in the oracle's secondary-ray generator (oracle/raygen.py).
RAYGEN_MUTANTS = [
    ("disk radius not square-rooted", [("rr, phi = np.sqrt(u1), 2 * np.pi * u2", "rr, phi = u1, 2 * np.pi * u2")]),
    ("uniform instead of cosine-weighted",
     [("        lx, ly, lz = rr * np.cos(phi), rr * np.sin(phi), np.sqrt(max(0.0, 1 - u1))\n",
       "        rr = np.sqrt(max(0.0, 1 - u1 * u1))\n        lx, ly, lz = rr * np.cos(phi), rr * np.sin(phi), u1\n")]),
    ("tangent basis sign", [("b2 = np.array([bb, sg_ + nrm[1] ** 2 * aa, -nrm[1]])",
                             "b2 = np.array([bb, sg_ + nrm[1] ** 2 * aa, nrm[1]])")]),
    ("normal not turned toward the ray", [("        if nrm @ din[i] > 0:\n", "        if nrm @ din[i] < 0:\n")]),
    ("offset without its factor 2", [("        off = offset_abs + 2.0 * l1 * 2.0 ** -L\n",
                                      "        off = offset_abs + l1 * 2.0 ** -L\n")]),
    ("pcg output shift", [("xs = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF", "xs = (((old >> 18) ^ old) >> 28) & 0xFFFFFFFF")]),
    ("pcg seed and sequence swapped", [("    state = (state + seed) & _MASK\n", "    state = (state + seq) & _MASK\n")]),
    ("mirror sign", [("d[i] = din[i] - 2.0 * (din[i] @ nrm) * nrm", "d[i] = din[i] + 2.0 * (din[i] @ nrm) * nrm")]),
    ("shadow ray not ended at the light", [("            tmax[i] = dist\n", "            tmax[i] = np.inf\n")]),
    ("shadow ray kept with the light behind", [("if dist > 0 and to_light @ nrm > 0:", "if dist > 0:")]),
]


def test_every_planted_mistake_in_the_ray_generator_fails_a_pin():
    src = open(os.path.join(ROOT, "oracle", "raygen.py")).read()

    def passes(text):
        m = _py_module(text, package="oracle")
        b = {"raygen": m, "shadow_rays": m.shadow_rays}
        return _py_pins_pass("test_oracle_raygen.py", b) and _py_pins_pass("test_oracle_shadow.py", b)
    assert passes(src), "the unchanged ray generator fails its pins in the harness"
    survivors = _survivors(src, RAYGEN_MUTANTS, passes)
    assert not survivors, f"planted mistakes in the ray generator that no pin catches: {survivors}"
