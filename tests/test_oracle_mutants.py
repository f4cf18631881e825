"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of the oracle (a flipped
comparison, a dropped term, a wrong index or sign, transposed operands), on
the CPU, and runs the oracle's pin tests against that copy: at least one pin
must fail.  The C oracle's copies are built with gcc into a temporary
directory and loaded through TM_ORACLE_LIB; the learned-model oracle's copies
replace ``oracle.cdf`` through TM_ORACLE_CDF.  The unmodified sources, run
the same way, must pass (the controls).  No GPU is used.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
MERGE_PINS = os.path.join(ROOT, "tests", "test_oracle_merge.py")
CDF_PINS = os.path.join(ROOT, "tests", "test_oracle_cdf.py")

# (name, file, text of the original, planted text).  The original text must
# occur exactly once in its file.
C_MUTANTS = [
    # rank primitives (Section 2)
    ("rank_low finds the high rank", "tm_oracle.c",
     "if (X[mid] < x) lo = mid + 1; else hi = mid;", "if (!(x < X[mid])) lo = mid + 1; else hi = mid;"),
    ("rank_high finds the low rank", "tm_oracle.c",
     "if (!(x < X[mid])) lo = mid + 1; else hi = mid;", "if (X[mid] < x) lo = mid + 1; else hi = mid;"),
    ("rank_low never returns len", "tm_oracle.c",
     "int64_t lo = 0, hi = len;          /* answer in [lo, hi] */", "int64_t lo = 0, hi = len > 0 ? len - 1 : 0;"),
    # block decomposition (Section 2)
    ("block start: floor for the long blocks", "tm_oracle.c",
     "if (i < r) return i * ceil_div(len, p);", "if (i < r) return i * (len / p);"),
    ("block start: remainder dropped", "tm_oracle.c",
     "return i * (len / p) + r;", "return i * (len / p);"),
    ("block start: one long block too few", "tm_oracle.c",
     "if (i < r) return i * ceil_div(len, p);", "if (i < r - 1) return i * ceil_div(len, p);"),
    ("block of: short blocks divided by the long size", "tm_oracle.c",
     "return (k - r * c) / (len / p) + r;", "return (k - r * c) / c + r;"),
    ("block of: remainder not added", "tm_oracle.c",
     "return (k - r * c) / (len / p) + r;", "return (k - r * c) / (len / p);"),
    # Steps 1-2
    ("xbar by rank_high", "tm_oracle.c",
     "xbar[i] = (xi < n) ? orc_rank_low_##S(A[xi], B, m) : m;",
     "xbar[i] = (xi < n) ? orc_rank_high_##S(A[xi], B, m) : m;"),
    ("ybar by rank_low", "tm_oracle.c",
     "ybar[j] = (yj < m) ? orc_rank_high_##S(B[yj], A, n) : n;",
     "ybar[j] = (yj < m) ? orc_rank_low_##S(B[yj], A, n) : n;"),
    ("empty A block ranked 0", "tm_oracle.c",
     "xbar[i] = (xi < n) ? orc_rank_low_##S(A[xi], B, m) : m;",
     "xbar[i] = (xi < n) ? orc_rank_low_##S(A[xi], B, m) : 0;"),
    ("xbar_p = n", "tm_oracle.c", "    xbar[p] = m;  ", "    xbar[p] = n;  "),
    # Steps 3-4: the five cases
    ("case (a) never taken", "tm_oracle.c", "if (xb == xb1) {", "if (xb == xb1 && 0) {"),
    ("case (e) never taken", "tm_oracle.c", "if (xb == yj) {", "if (xb == yj && 0) {"),
    ("case (e) runs to the block end", "tm_oracle.c",
     "row[0] = xi; row[1] = bar_oth[j]; row[2] = xb;", "row[0] = xi; row[1] = xi1; row[2] = xb;"),
    ("case (b) also for neighbouring blocks", "tm_oracle.c", "if (j1 == j) {", "if (j1 == j || j1 == j + 1) {"),
    ("case (c) own range to the block end", "tm_oracle.c",
     "row[0] = xi; row[1] = bar_oth[j + 1];", "row[0] = xi; row[1] = xi1;"),
    ("case (c) other range to the next cross rank", "tm_oracle.c",
     "row[3] = yj1; row[4] = c0; row[5] = 'c';", "row[3] = xb1; row[4] = c0; row[5] = 'c';"),
    ("case (c)/(d) test inverted", "tm_oracle.c", "if (xb1 != yj1) {", "if (xb1 == yj1) {"),
    ("case (d) as printed (x_{j+1})", "tm_oracle.c",
     "row[0] = xi; row[1] = xi1; row[2] = xb; row[3] = yj1; row[4] = c0; row[5] = 'd';",
     "row[0] = xi; row[1] = orc_block_start(len_own, p, j + 1); row[2] = xb; row[3] = yj1; row[4] = c0; "
     "row[5] = 'd';"),
    ("next other block start from the wrong block", "tm_oracle.c",
     "int64_t yj1 = orc_block_start(len_oth, p, j + 1);", "int64_t yj1 = orc_block_start(len_oth, p, j1);"),
    ("output offset from the next cross rank", "tm_oracle.c",
     "int64_t c0  = xi + xb;", "int64_t c0  = xi + xb1;"),
    ("Step 4 with the cross ranks not exchanged", "tm_oracle.c",
     "one_side_case(m, n, p, k - p, ybar, xbar, row);", "one_side_case(m, n, p, k - p, xbar, ybar, row);"),
    ("B-side subproblems merged B first", "tm_oracle.c",
     "orc_merge_two_pointer_##S(A + row[2], Av + row[2], row[3] - row[2],       \\\n"
     "                                      B + row[0], Bv + row[0], row[1] - row[0],       \\",
     "orc_merge_two_pointer_##S(B + row[0], Bv + row[0], row[1] - row[0],       \\\n"
     "                                      A + row[2], Av + row[2], row[3] - row[2],       \\"),
    # merges
    ("two-pointer takes B on ties", "tm_oracle.c",
     "if (B[j] < A[i]) { C[k] = B[j];", "if (!(A[i] < B[j])) { C[k] = B[j];"),
    ("two-pointer drops the B tail", "tm_oracle.c",
     "while (j < m) { C[k] = B[j]; Cv[k] = Bv[j]; ++j; ++k; }", "while (0) { }"),
    ("two-pointer moves the wrong payload", "tm_oracle.c",
     "else             { C[k] = A[i]; Cv[k] = Av[i]; ++i; }",
     "else             { C[k] = A[i]; Cv[k] = Av[k < n ? k : i]; ++i; }"),
    ("rank scatter places A by rank_high", "tm_oracle.c",
     "int64_t pos = i + orc_rank_low_##S(A[i], B, m);", "int64_t pos = i + orc_rank_high_##S(A[i], B, m);"),
    ("rank scatter places B by rank_low", "tm_oracle.c",
     "int64_t pos = j + orc_rank_high_##S(B[j], A, n);", "int64_t pos = j + orc_rank_low_##S(B[j], A, n);"),
    ("batched merge skips the first pair", "tm_oracle.c",
     "for (int64_t k = 0; k < pairs; ++k) {", "for (int64_t k = 1; k < pairs; ++k) {"),
    ("batched merge forgets the B offset", "tm_oracle.c",
     "C + a0 + b0, Cv + a0 + b0);", "C + a0, Cv + a0);"),
    # merge sort (Section 3)
    ("run sort not stable", "tm_oracle.c",
     "while (b > lo && k < keys[b - 1]) {", "while (b > lo && !(keys[b - 1] < k)) {"),
    ("unpaired last run not carried", "tm_oracle.c",
     "for (int64_t lo = 0; lo < n; lo += 2 * w) {", "for (int64_t lo = 0; lo + w < n; lo += 2 * w) {"),
    ("result left in the scratch buffer", "tm_oracle.c", "if (sk != keys) {", "if (0) {"),
    # the threaded CPU baseline
    ("threaded: B-side subproblems skipped", "paper_parallel.c",
     "for (int64_t k = g->t; k < 2 * p; k += g->threads) {", "for (int64_t k = g->t; k < p; k += g->threads) {"),
    ("threaded: ybar by rank_low", "paper_parallel.c",
     "g->ybar[i] = (yi < m) ? orc_rank_high_##S(g->B[yi], g->A, n) : n;",
     "g->ybar[i] = (yi < m) ? orc_rank_low_##S(g->B[yi], g->A, n) : n;"),
    ("threaded: ybar_p = m", "paper_parallel.c", "    ybar[p] = n;  ", "    ybar[p] = m;  "),
]

CDF_MUTANTS = [
    ("knot ranks rounded up", "(s * N) // S", "(s * N + S - 1) // S"),
    ("last knot one short of the end", "K[S] = X[N - 1]", "K[S] = X[N - 2]"),
    ("segment counts knots below q only", "if K[mid] <= q:", "if K[mid] < q:"),
    ("position in segment not clamped", "t = np.clip(t, 0.0, 1.0)", "t = t"),
    ("segment feature off by half a segment", "f1 = (2.0 * s + 1.0) / S - 1.0", "f1 = (2.0 * s) / S - 1.0"),
    ("no interpolation inside a segment", "pla = Rs + t * seg", "pla = Rs + 0.0 * seg"),
    ("no ReLU in the forward pass", "h = np.maximum(z, 0.0)", "h = z"),
    ("no ReLU mask in the backward pass", "dz = np.outer(dy, params[\"w2\"]) * (fw[\"z\"] > 0)",
     "dz = np.outer(dy, params[\"w2\"])"),
    ("loss without the half", "loss = 0.5 * float(np.mean(r * r))", "loss = float(np.mean(r * r))"),
    ("residual gradient sign", "dy = r / B ", "dy = -r / B "),
    ("target sign", "tau = (np.asarray(L, dtype=np.float64) - fw[\"pla\"]) / fw[\"scale\"]\n    r = fw",
     "tau = (fw[\"pla\"] - np.asarray(L, dtype=np.float64)) / fw[\"scale\"]\n    r = fw"),
    ("features transposed in dW1", "    F = np.stack([fw[\"f0\"], fw[\"f1\"]], axis=1)\n",
     "    F = np.stack([fw[\"f1\"], fw[\"f0\"]], axis=1)\n"),
    ("bias gradient dropped", "db2 = np.sum(dy)", "db2 = 0.0 * np.sum(dy)"),
    ("Adam without bias correction of m", "mhat = m / (1.0 - BETA1 ** k)", "mhat = m"),
    ("Adam second moment of g, not g^2", "(1.0 - BETA2) * g * g", "(1.0 - BETA2) * g"),
    ("error bound without the absolute value", "np.max(np.abs(fw[\"y\"] - tau))", "np.max(fw[\"y\"] - tau)"),
]


def _read(path):
    with open(path) as f:
        return f.read()


def _plant(text, old, new, what):
    assert text.count(old) == 1, f"{what}: the original text must occur exactly once"
    return text.replace(old, new)


def _run_pins(pins, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def _build_c(tmp, name, sources):
    paths = []
    for fname, text in sources.items():
        path = os.path.join(tmp, fname)
        with open(path, "w") as f:
            f.write(text)
        paths.append(path)
    lib = os.path.join(tmp, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-pthread", "-o", lib] + paths)
    return lib


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Runs every planted copy (and the controls) once, in parallel."""
    base = {f: _read(os.path.join(ORACLE, f)) for f in ("tm_oracle.c", "paper_parallel.c")}
    cdf_src = _read(os.path.join(ORACLE, "cdf.py"))
    jobs = {}
    tmp = tmp_path_factory.mktemp("mutants")

    def c_job(idx, name, fname=None, old=None, new=None):
        d = os.path.join(tmp, f"c{idx}")
        os.makedirs(d)
        srcs = dict(base)
        if fname is not None:
            srcs[fname] = _plant(srcs[fname], old, new, name)
        lib = _build_c(d, f"m{idx}", srcs)
        return _run_pins(MERGE_PINS, {"TM_ORACLE_LIB": lib})

    def cdf_job(idx, name, old=None, new=None):
        d = os.path.join(tmp, f"p{idx}")
        os.makedirs(d)
        path = os.path.join(d, "cdf.py")
        with open(path, "w") as f:
            f.write(cdf_src if old is None else _plant(cdf_src, old, new, name))
        return _run_pins(CDF_PINS, {"TM_ORACLE_CDF": path})

    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        jobs["control: C oracle"] = ex.submit(c_job, 0, "control")
        jobs["control: cdf oracle"] = ex.submit(cdf_job, 0, "control")
        for k, (name, fname, old, new) in enumerate(C_MUTANTS, 1):
            jobs[name] = ex.submit(c_job, k, name, fname, old, new)
        for k, (name, old, new) in enumerate(CDF_MUTANTS, 1):
            jobs[name] = ex.submit(cdf_job, k, name, old, new)
        return {name: fut.result() for name, fut in jobs.items()}


@pytest.mark.parametrize("name", ["control: C oracle", "control: cdf oracle"])
def test_unplanted_oracle_passes_its_pins(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in C_MUTANTS] + [m[0] for m in CDF_MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    # 1: a pin failed.  A crash of the planted copy would also show the
    # mistake, but every case here is chosen to fail an assertion instead.
    what = "crashed the pins" if rc < 0 else "survived the pins"
    assert rc == 1, f"planted mistake '{name}' {what} (pytest exit {rc}):\n{tail}"
