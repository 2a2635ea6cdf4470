"""The oracle's pins catch planted mistakes (CPU only).

Each case copies ``oracle/`` into a temporary directory, plants one plausible
mistake in the copy (a transposed operand, a dropped term, a wrong sign or
index, alpha and beta swapped, a wrong stack cut, a dropped slice level, ...),
builds it, and runs every pin test of ``test_oracle_pins.py``,
``test_oracle_ozaki_pins.py``, ``test_oracle_fp32_pins.py`` and the hand-worked
fixtures of ``test_golden.py`` against the copy in a child process. The mistake must make at least one pin fail. The unchanged
copy must pass them all, which shows that the child really runs the copy.

Every planted mistake keeps all memory accesses inside their buffers (a changed
index stays within the same block), so a mistake shows up as a wrong value, not
as a crash. Each replacement must match the source exactly once: when the
oracle's text changes, the test fails and names the mutant to update.
"""
import importlib.util
import inspect
import os
import shutil
import subprocess
import sys
import traceback
from concurrent.futures import ThreadPoolExecutor

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PIN_MODULES = ("test_oracle_pins.py", "test_oracle_ozaki_pins.py", "test_oracle_fp32_pins.py", "test_golden.py")

C_SRC = "dbcsr_oracle.c"
PY_SRC = "oracle.py"

# (name, file in oracle/, text in the source, replacement)
MUTANTS = [
    # ---- the block product of Sec. II (mode 0: plain FP64)
    ("A block read transposed", C_SRC,
     "sum = sum + ablk[r + (int64_t)l * m] * bblk[l + (int64_t)cc * kk];",
     "sum = sum + ablk[l + (int64_t)r * kk] * bblk[l + (int64_t)cc * kk];"),
    ("B block read transposed", C_SRC,
     "sum = sum + ablk[r + (int64_t)l * m] * bblk[l + (int64_t)cc * kk];",
     "sum = sum + ablk[r + (int64_t)l * m] * bblk[cc + (int64_t)l * n];"),
    ("last inner term dropped", C_SRC,
     "for (int l = 0; l < kk; l++)\n                                    sum = sum + ablk",
     "for (int l = 0; l < kk - 1; l++)\n                                    sum = sum + ablk"),
    ("inner index summed descending", C_SRC,
     "for (int l = 0; l < kk; l++)\n                                    sum = sum + ablk",
     "for (int l = kk - 1; l >= 0; l--)\n                                    sum = sum + ablk"),
    ("old accumulator not carried between k blocks", C_SRC,
     "double sum = x[r + (int64_t)cc * m];",
     "double sum = 0.0;"),
    ("product and sum fused into one rounding (FMA)", C_SRC,
     "sum = sum + ablk[r + (int64_t)l * m] * bblk[l + (int64_t)cc * kk];",
     "sum = fma(ablk[r + (int64_t)l * m], bblk[l + (int64_t)cc * kk], sum);"),
    ("alpha and beta swapped", C_SRC,
     "double r = alpha * v;\n                    if (old) r = r + beta * old[e];",
     "double r = beta * v;\n                    if (old) r = r + alpha * old[e];"),
    ("sign of the beta term", C_SRC,
     "if (old) r = r + beta * old[e];",
     "if (old) r = r - beta * old[e];"),
    ("old C read when beta = 0", C_SRC,
     "int use_old = (beta != 0.0) && C && C->nblks > 0;",
     "int use_old = C && C->nblks > 0;"),
    ("old C pattern dropped", C_SRC,
     "    if (use_old)\n        for (int64_t q = cold->rowptr[i];",
     "    if (0)\n        for (int64_t q = cold->rowptr[i];"),
    ("op() block copied without transposing", C_SRC,
     "dst[x + (int64_t)y * sc] = src[y + (int64_t)x * sr];",
     "dst[x + (int64_t)y * sc] = src[x + (int64_t)y * sc];"),
    ("duplicate blocks accepted", C_SRC,
     "free(order); free(off); rows_free(v); return -1;   /* duplicate */",
     "(void)0;"),
    ("inner block sizes not checked", C_SRC,
     "if (a.cs[k] != b.rs[k]) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }",
     "if (0) { rows_free(&a); rows_free(&b); rows_free(&c); return -2; }"),
    # ---- double-double accumulation (Dot2)
    ("Dot2: TwoSum error dropped", C_SRC,
     "sl = sl + (pe + te);",
     "sl = sl + pe;"),
    ("Dot2: TwoProduct error dropped", C_SRC,
     "sl = sl + (pe + te);",
     "sl = sl + te;"),
    ("Dot2: compensation not added at the end", C_SRC,
     "double v = (mode == 1) ? acc[j][e] + cmp[j][e] : acc[j][e];",
     "double v = acc[j][e];"),
    # ---- single precision (mode 2)
    ("FP32: inputs not rounded to FP32", C_SRC,
     "float pa = (float)ablk[r + (int64_t)l * m];\n"
     "                                    float pb = (float)bblk[l + (int64_t)cc * kk];\n"
     "                                    float pr = pa * pb;",
     "double pa = ablk[r + (int64_t)l * m];\n"
     "                                    double pb = bblk[l + (int64_t)cc * kk];\n"
     "                                    float pr = (float)(pa * pb);"),
    ("FP32: product kept in FP64", C_SRC,
     "float pr = pa * pb;\n                                    sum = sum + pr;",
     "double pr = (double)pa * pb;\n                                    sum = (float)(sum + pr);"),
    # ---- stack list (Sec. II: Traversal + Generation)
    ("stack cut one entry late", C_SRC,
     "if (newshape || run == stack_cap)",
     "if (newshape || run == stack_cap + 1)"),
    ("stack counter not reset at a new shape", C_SRC,
     "if (newshape || run == stack_cap) { sid++; run = 0; }",
     "if (newshape || run == stack_cap) { sid++; if (!newshape) run = 0; }"),
    ("stack shape written as (m, k, n)", C_SRC,
     "x[1] = a.rs[i]; x[2] = b.cs[j]; x[3] = a.cs[k];",
     "x[1] = a.rs[i]; x[2] = a.cs[k]; x[3] = b.cs[j];"),
    ("new stack not started when only k changes", C_SRC,
     "|| x[2] != x[2 - 7] || x[3] != x[3 - 7];",
     "|| x[2] != x[2 - 7];"),
    ("stack entries ordered k before j", C_SRC,
     "x[4] = i; x[5] = j; x[6] = k;",
     "x[4] = i; x[5] = k; x[6] = j;"),
    # ---- dense GEMM (Sec. III)
    ("dense GEMM: op(A) = T ignored", C_SRC,
     "double x = trA ? A[l + r * lda] : A[r + l * lda];",
     "double x = A[r + l * lda];"),
    ("dense GEMM: sign of the beta term", C_SRC,
     "if (beta != 0.0) v = v + beta * C[r + c * ldc];\n            C[r + c * ldc] = v;",
     "if (beta != 0.0) v = v - beta * C[r + c * ldc];\n            C[r + c * ldc] = v;"),
    # ---- Ozaki slices
    ("slices rounded instead of truncated", C_SRC,
     "double sg = trunc(ldexp(r, 7 * t));",
     "double sg = round(ldexp(r, 7 * t));"),
    ("slice width 6 bits in the remainder", C_SRC,
     "r = r - ldexp(sg, -7 * t);",
     "r = r - ldexp(sg, -6 * t);"),
    ("exponent one too small", C_SRC,
     "(void)frexp(mu, &e);\n    return e;",
     "(void)frexp(mu, &e);\n    return e - 1;"),
    ("row maximum taken as its last element", C_SRC,
     "else if (v > mu) mu = v;",
     "else mu = v;"),
    ("dense GEMM: product and sum fused (FMA)", C_SRC,
     "s = s + x * y;",
     "s = fma(x, y, s);"),
    ("column maximum taken as its last element", C_SRC,
     "else if (v > nu) nu = v;",
     "else nu = v;"),
    ("level s + 1 dropped", C_SRC,
     "for (int u = 1; u + t <= s + 1; u++) {",
     "for (int u = 1; u + t <= s; u++) {"),
    ("level weight off by one slice", C_SRC,
     "S += (__int128)G[(size_t)d * N + j] << (7 * (s + 1 - d));",
     "S += (__int128)G[(size_t)d * N + j] << (7 * (s + 2 - d));"),
    ("recombined in FP64 term by term", C_SRC,
     "__int128 S = 0;",
     "double S = 0;"),
    ("column exponent subtracted", C_SRC,
     "e_row[i] + f_col[j] - 7 * (s + 1)",
     "e_row[i] - f_col[j] - 7 * (s + 1)"),
    ("Ozaki: old C read when beta = 0", C_SRC,
     "if (beta != 0.0) v = v + beta * C[i + j * ldc];",
     "v = v + beta * C[i + j * ldc];"),
    ("non-finite row of A not marked NaN", C_SRC,
     "if (e_row[i] == OZ_NONFINITE || f_col[j] == OZ_NONFINITE) {",
     "if (f_col[j] == OZ_NONFINITE) {"),
    ("non-finite column of B not marked NaN", C_SRC,
     "if (e_row[i] == OZ_NONFINITE || f_col[j] == OZ_NONFINITE) {",
     "if (e_row[i] == OZ_NONFINITE) {"),
    ("subnormal result rounded twice (53 bits, then at 2^-1074)", C_SRC,
     "if (n - 1 + k < -1022) drop = -1074 - k;",
     "if (0) drop = -1074 - k;"),
    ("rounding tie broken away from zero", C_SRC,
     "if (rem > half || (rem == half && (q & 1))) q += 1;",
     "if (rem >= half) q += 1;"),
    # ---- Python helpers of the oracle
    ("densify: block placed at the transposed corner", PY_SRC,
     "D[ro[i]:ro[i] + m, co[j]:co[j] + n] = np.asarray(M.data[pos:pos + m * n]).reshape((m, n), order=\"F\")",
     "D[ro[i]:ro[i] + m, co[j]:co[j] + n] = np.asarray(M.data[pos:pos + m * n]).reshape((m, n), order=\"C\")"),
    ("TF32: rounding bit at the wrong place", PY_SRC,
     "r = (mag + np.uint32(0x1000)) & np.uint32(0xFFFFE000)",
     "r = (mag + np.uint32(0x0FFF)) & np.uint32(0xFFFFE000)"),
    ("normwise error without the norm of B", PY_SRC,
     "den = np.linalg.norm(Ad) * np.linalg.norm(Bd)",
     "den = np.linalg.norm(Ad)"),
]


# --------------------------------------------------------------------------
# child process: run every pin against the oracle found first on sys.path
# --------------------------------------------------------------------------
def _pin_cases(mod):
    fns = [(name, fn) for name, fn in vars(mod).items()
           if name.startswith("test_") and inspect.isfunction(fn)]
    fns.sort(key=lambda t: inspect.getsourcelines(t[1])[1])
    for name, fn in fns:
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            yield name, fn, {}
            continue
        assert len(marks) == 1, f"{name}: one parametrize mark expected"
        argnames, argvalues = marks[0].args[:2]
        names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
        for v in argvalues:
            vals = tuple(v) if len(names) > 1 else (v,)
            yield f"{name}[{'-'.join(map(str, vals))}]", fn, dict(zip(names, vals))


def _child(copy_dir):
    sys.path[:0] = [copy_dir, ROOT]
    import oracle
    assert os.path.dirname(os.path.abspath(oracle.__file__)) == os.path.join(copy_dir, "oracle")
    failed, passed = [], 0
    for fname in PIN_MODULES:
        spec = importlib.util.spec_from_file_location(fname[:-3], os.path.join(HERE, fname))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        for name, fn, kw in _pin_cases(mod):
            try:
                fn(**kw)
                passed += 1
            except pytest.skip.Exception:
                pass
            except (Exception, pytest.fail.Exception):   # a failed assertion or pytest.raises
                failed.append(name)
    print(f"PASSED {passed}")
    for name in failed:
        print(f"FAILED {name}")


# --------------------------------------------------------------------------
# parent: copy, mutate, build (in the child), collect
# --------------------------------------------------------------------------
def _prepare(base, tag, mutant):
    copy_dir = os.path.join(base, tag)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(copy_dir, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    if mutant is not None:
        _, fname, old, new = mutant
        path = os.path.join(copy_dir, "oracle", fname)
        with open(path) as f:
            src = f.read()
        assert src.count(old) == 1, f"mutant {mutant[0]!r}: its text occurs {src.count(old)} times in {fname}"
        with open(path, "w") as f:
            f.write(src.replace(old, new))
    return copy_dir


def _run(copy_dir):
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    p = subprocess.run([sys.executable, os.path.abspath(__file__), copy_dir], cwd=copy_dir, env=env,
                       capture_output=True, text=True, timeout=600)
    passed = [int(l.split()[1]) for l in p.stdout.splitlines() if l.startswith("PASSED ")]
    failed = [l[len("FAILED "):] for l in p.stdout.splitlines() if l.startswith("FAILED ")]
    return p.returncode, passed[0] if passed else None, failed, p.stderr[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = str(tmp_path)
    jobs = [("control", None)] + [(f"m{q:02d}", m) for q, m in enumerate(MUTANTS)]
    dirs = {tag: _prepare(base, tag, m) for tag, m in jobs}
    with ThreadPoolExecutor(max_workers=4) as ex:
        results = dict(zip(dirs, ex.map(_run, dirs.values())))

    rc, passed, failed, err = results["control"]
    assert rc == 0 and passed and not failed, f"unchanged oracle copy: rc={rc} failed={failed}\n{err}"

    survivors = []
    for tag, m in jobs[1:]:
        rc, passed, failed, err = results[tag]
        assert rc == 0 and passed is not None, f"mutant {m[0]!r} did not run: rc={rc}\n{err}"
        if not failed:
            survivors.append(m[0])
    assert not survivors, f"planted mistakes no pin detects: {survivors}"


if __name__ == "__main__":
    try:
        _child(sys.argv[1])
    except Exception:
        traceback.print_exc()
        sys.exit(1)
