"""Planted mistakes in the oracle are caught by its pins.

The oracle is trusted because tests pin it to things it does not compute
itself (brute force, exact rationals, the lattice of Eq. (2)).  This file
checks that those pins are strong enough: each mutant below is a copy of
oracle/msp_oracle.c with one plausible mistake -- a dropped term, a wrong
sign or index, a misread reading -- compiled to a temporary library.  A
child process runs a fast selection of the pins against it, and every
mutant must fail at least one of them, while the unmodified source passes
all of them.  Nothing here touches the product path or a GPU.
"""
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "msp_oracle.c")

# (name, function the change is made in, text, replacement): the first
# occurrence of the text after the start of that function is replaced.
# Every mutant ends within seconds (a partial norm that drops rho_{t+1}
# instead of doubling it would also be wrong, but its tree never stops
# growing, so it is not used here).
MUTANTS = [
    ("centre from the transposed mu entry", "static double center(",
     "e->mu[(size_t)i * e->dd + t]", "e->mu[(size_t)t * e->dd + i]"),
    ("centre of the wrong sign", "static void enum_level(",
     "const double cstar = -y;", "const double cstar = y;"),
    ("partial norm with rho_{t+1} counted twice", "static void enum_level(",
     "fma(xx, e->B[t], rho_p)", "fma(xx, e->B[t], 2.0 * rho_p)"),
    ("w updated from the wrong row of bhat", "static void enum_level(",
     "e->bhat[(size_t)t * dim + c]", "e->bhat[(size_t)(t - 1) * dim + c]"),
    ("l1 norm without the absolute value", "static double norm1(",
     "fabs(w[c])", "w[c]"),
    ("zig-zag starting on the wrong side", "static void enum_level(",
     "int s = (cstar >= (double)u1) ? 1 : -1;", "int s = (cstar >= (double)u1) ? -1 : 1;"),
    ("one-direction phase walking back past the centre", "static void enum_level(",
     "dir = (u > u1) ? 1 : -1;", "dir = (u > u1) ? -1 : 1;"),
    ("next() skipping every other value", "static void enum_level(",
     "else { zi += 1; u = zigzag(u1, s, zi); }", "else { zi += 2; u = zigzag(u1, s, zi); }"),
    ("leaf without sign normalisation", "static int leaf_check(",
     "if (last == -rmax)", "if (0 && last == -rmax)"),
    ("no slack on the bounds", "int oracle_enumerate_bounds(",
     "e.eps = o->use_eps ? R * 0x1p-20 : 0.0;", "e.eps = 0.0;"),
    ("Lovasz test with a smaller delta", "static int lll_core(",
     "if (B[k] < rhs)", "if (B[k] < 0.5 * rhs)"),
    ("size reduction updating mu with the wrong sign", "static int lll_core(",
     "fma(-qd, mu", "fma(qd, mu"),
    ("Gram-Schmidt mu divided by the first B", "int oracle_gso(",
     "mu[(size_t)i * dd + j] = acc / B[j];", "mu[(size_t)i * dd + j] = acc / B[0];"),
    ("lattice with +N d in the first column", "int oracle_build_lattice_bounds(",
     "i128 v = -(i128)N * (i128)d[i];", "i128 v = (i128)N * (i128)d[i];"),
    ("rank discrepancy counted from one", "static int value_cost(",
     "e->o.lds_rank ? (int)pos", "e->o.lds_rank ? (int)pos + 1"),
    ("flat discrepancy counting only values above the first", "static int value_cost(",
     "(u != u1)", "(u > u1)"),
    ("block search centred with the wrong sign", "static void svp_level(",
     "cstar = -y;", "cstar = y;"),
    ("split prefix recorded with the parent's partial norm", "static void enum_level(",
     "e->pre_rho[p] = rho;", "e->pre_rho[p] = rho_p;"),
    ("extraction testing one row too few", "int oracle_extract(",
     "for (int i = 0; i < m; ++i) if (b[i] != 0)", "for (int i = 0; i < m - 1; ++i) if (b[i] != 0)"),
    ("bounded lattice without c_j on the diagonal", "int oracle_build_lattice_bounds(",
     "b[m + (j - 1)] = 2 * (rmax / (r ? r[j - 1] : 1));", "b[m + (j - 1)] = 2;"),
    ("l1 lane tree missing its last combine", "static double norm1(",
     "for (int off = G / 2; off >= 1; off /= 2)", "for (int off = G / 2; off > 1; off /= 2)"),
    ("discrepancy leaves reported below the budget", "static void enum_level(",
     "disc + cost == e->o.lds", "disc + cost <= e->o.lds"),
    ("leaf without the range check on v", "static int leaf_check(",
     "if (v[c] > rmax || v[c] < -rmax || (v[c] + rmax) % cc != 0) return 0;",
     "if ((v[c] + rmax) % cc != 0) return 0;"),
    ("bhat rows adding the projections instead of subtracting them", "int oracle_gso(",
     "acc = fma(-mu[(size_t)i * dd + j], bhat", "acc = fma(mu[(size_t)i * dd + j], bhat"),
    ("subtree start rebuilding rho from its last level only", "int oracle_enumerate_bounds(",
     "rho0 = fma(xx, B[t], rho0);", "rho0 = fma(xx, B[t], 0.0);"),
    ("walk position of a prefix value off by one", "static long level_position(",
     "if (u == target) return pos;", "if (u == target) return pos + 1;"),
    ("BKZ insertion step dropping the Bezout term of the first row", "int oracle_bkz(",
     "const i128 v1 = -(i128)tb * c0[c] + (i128)sa * c1[c];", "const i128 v1 = (i128)sa * c1[c];"),
    ("filter-only Hoelder mode cutting like the default", "static void enum_level(",
     "if (fail && e->o.hoelder == HOELDER_CUT) {", "if (fail && e->o.hoelder != HOELDER_OFF) {"),
    ("Hoelder failure still expanded", "static void enum_level(",
     "if (!fail) {", "if (1) {"),
    ("first-solution mode whose stop does not reach the levels above", "static void enum_level(",
     "if (e->s.stopped) return;", "if (0) return;"),
    ("literal mode normalising the sign at the leaf", "static int leaf_check(",
     "    if (e->o.sym) {", "    if (1) {"),
    ("reduction's mu scaled by the row's own reciprocal", "static void gso_row(",
     "mu[(size_t)k * K + j] = acc * invB[j];", "mu[(size_t)k * K + j] = acc * invB[k];"),
    ("LLL swap leaving the Gram matrix's columns in place", "static int lll_core(",
     "for (int i = 0; i < K; ++i) {      /* swap columns k-1, k of G */",
     "for (int i = 0; i < 0; ++i) {      /* swap columns k-1, k of G */"),
    ("Lovasz test reading mu of the row above", "static int lll_core(",
     "double mk = mu[(size_t)k * K + (k - 1)];", "double mk = mu[(size_t)(k - 1) * K + (k > 1 ? k - 2 : 0)];"),
    ("bounded leaf without the per-variable scale c_j", "static int leaf_check(",
     "const int64_t cc = 2 * (rmax / (e->r ? e->r[c] : 1));", "const int64_t cc = 2 * rmax;"),
]


def mutate(src, where, old, new):
    start = src.index(where)
    at = src.index(old, start)
    return src[:at] + new + src[at + len(old):]


def compile_library(source_text, out_dir, tag):
    """The oracle's own build flags (oracle/build.py) on a copy of the source."""
    c = os.path.join(out_dir, f"{tag}.c")
    so = os.path.join(out_dir, f"{tag}.so")
    with open(c, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", so, c, "-lm"], check=True, capture_output=True)
    return so


# --------------------------------------------------------------------------
# child process: the pins, run against the library at sys.argv[1]

def _pins():
    import numpy as np

    from oracle import definition as DEF
    from oracle import oracle as O
    import test_oracle_counts as TC
    import test_oracle_enum as TE
    import test_oracle_lattice as TL

    def sets():
        """solution sets equal brute force (1 and 8 lanes; all pruning modes)"""
        for k, inst in enumerate(TE.SMALL[:12]):
            want = DEF.brute_force(inst.A, inst.d)
            for lanes in (1, 8):
                got = O.solve(inst.A, inst.d, lanes=lanes).result.solutions
                assert np.array_equal(got, want), (k, lanes)
            for hoelder, sym in TE.MODES[1:]:
                got = O.solve(inst.A, inst.d, hoelder=hoelder, sym=sym).result.solutions
                assert np.array_equal(got, want), (k, hoelder, sym)

    def lattice():
        for c in TL.CASES:
            TL.test_lattice_contains_planted_solution(c)
            TL.test_extraction_is_a_kernel_basis(c)

    def lll():
        for c in TL.CASES:
            TL.test_lll_is_unimodular_and_reduced(c)

    def gso():
        for c in TL.CASES:
            TL.test_gso_against_exact_rationals(c)

    def counts():
        for inst in TC.CASES[:3]:
            for sym in (False, True):
                for mode in (O.HOELDER_OFF, O.HOELDER_FILTER):
                    TC.test_counts_equal_the_definition(inst, sym, mode)

    def split():
        for inst in TC.CASES[:2]:
            for sym in (False, True):
                TC.test_split_prefixes_and_their_norms_are_exact(inst, sym)
        for k in (1, 3, 6):
            TE.test_split_is_a_partition(TE.SMALL[1], k)
        TE.test_first_mode_returns_a_valid_solution()
        for k in (0, 1, 2):
            TE.test_first_mode_stops_at_one_of_many(k)

    def lds():
        import test_oracle_lds as TD
        for rank in (False, True):
            for inst in TD.CASES[:3]:
                TD.test_iterations_partition_the_solution_set(inst, rank)
            TD.test_first_solution_comes_at_the_least_discrepancy(rank)
            for k, depth in ((1, 3), (2, 5), (4, 6)):
                TD.test_split_iteration_is_a_partition(TD.CASES[1], k, depth, rank)

    def bkz():
        import test_oracle_bkz as TB
        TB.test_same_lattice_and_volume(TB.CASES[0], 4)
        for inst in TB.CASES[:2]:
            TB.test_blocks_are_reduced(inst)
        TB.test_full_block_gives_a_shortest_vector()
        for inst in TB.HARD:
            TB.test_same_lattice_and_volume(inst, 4)
            TB.test_block_search_repairs_what_lll_leaves(inst)
            TB.test_full_block_finds_the_shortest_vector_lll_missed(inst)

    def bounds():
        import test_oracle_bounds as TN
        TN.test_lattice_columns()
        for inst in TN.CASES[:3]:
            TN.test_bounded_solution_sets_equal_brute_force(inst, O.HOELDER_CUT, True)

    return {"sets": sets, "lattice": lattice, "lll": lll, "gso": gso, "counts": counts, "split": split, "lds": lds, "bkz": bkz,
            "bounds": bounds}


def child_main(lib_path, stop_at_first=True):
    """Runs the pins in order; a mutant stops at its first failure (a wrong
    table can make a later, larger search run very long)."""
    from oracle import build as OB
    from oracle import oracle as O
    OB.build = lambda force=False: lib_path
    O._lib = None
    out = {}
    for name, fn in _pins().items():
        try:
            fn()
            out[name] = "pass"
        except (KeyboardInterrupt, SystemExit):
            raise
        except BaseException as e:   # assertion, oracle error, pytest outcome
            out[name] = f"fail: {type(e).__name__}: {str(e)[:160]}"
            if stop_at_first:
                break
    print(json.dumps(out), flush=True)


CHILD = ("import sys; sys.path[:0] = [{root!r}, {tests!r}]; "
         "import test_oracle_mutations as t; t.child_main(sys.argv[1])").format(
    root=ROOT, tests=os.path.join(ROOT, "tests"))


# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    out_dir = str(tmp_path_factory.mktemp("mutants"))
    src = open(SRC).read()
    jobs = [("unmodified", src)] + [(name, mutate(src, where, old, new)) for name, where, old, new in MUTANTS]

    def run(job):
        i, (name, text) = job
        so = compile_library(text, out_dir, f"oracle{i}")
        try:
            r = subprocess.run([sys.executable, "-c", CHILD, so], capture_output=True, text=True, timeout=300,
                               cwd=ROOT)
        except subprocess.TimeoutExpired:
            return name, {"run": "fail: timed out"}
        if r.returncode != 0:
            return name, {"run": f"fail: exit {r.returncode}: {r.stderr[-200:]}"}
        return name, json.loads(r.stdout.strip().splitlines()[-1])

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(run, enumerate(jobs)))


def test_mutations_apply_once_inside_their_function():
    src = open(SRC).read()
    for name, where, old, new in MUTANTS:
        assert src.count(where) == 1, name
        start = src.index(where)
        nxt = src.find("\n}\n", start)      # end of that function
        assert start < src.index(old, start) < nxt, name


def test_the_unmodified_oracle_passes_every_pin(outcomes):
    res = outcomes["unmodified"]
    assert res and all(v == "pass" for v in res.values()), res


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_each_planted_mistake_fails_a_pin(outcomes, name):
    res = outcomes[name]
    assert any(v != "pass" for v in res.values()), res


# --------------------------------------------------------------------------
# The scorer's CPU reference (oracle/mlp.py): planted mistakes in copies of
# the module, each loaded in place of the original for the scorer's pins.

MLP_SRC = os.path.join(ROOT, "oracle", "mlp.py")

MLP_MUTANTS = [
    ("BCE gradient of the wrong sign",
     "(1.0 / (1.0 + np.exp(-z)) - f)", "(f - 1.0 / (1.0 + np.exp(-z)))"),
    ("node-term gradient without the factor 2",
     "dy[:, 1] = 2.0 * NODE_WEIGHT * diff / B", "dy[:, 1] = NODE_WEIGHT * diff / B"),
    ("backward without the second ReLU's mask",
     "dh2 = (dyr @ r(p[\"W3\"]).T) * (c[\"a2\"] > 0)", "dh2 = (dyr @ r(p[\"W3\"]).T)"),
    ("W2 gradient transposed",
     "g[\"W2\"] = c[\"h1b\"].T @ dh2r", "g[\"W2\"] = (c[\"h1b\"].T @ dh2r).T"),
    ("b1 gradient taken from the second layer",
     "g[\"b1\"] = dh1.sum(axis=0)", "g[\"b1\"] = dh2.sum(axis=0)"),
    ("pos_weight on the rows without a solution",
     "np.where(f > 0.5, pos_weight, 1.0)", "np.where(f > 0.5, 1.0, pos_weight)"),
    ("bfloat16 rounding with ties away from zero",
     "r = ((u + 0x7FFF + lsb) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16"),
    ("forward without the second bias",
     "a2 = h1b @ r(p[\"W2\"]) + p[\"b2\"]", "a2 = h1b @ r(p[\"W2\"])"),
    ("node term weighted 0.2 (loss and gradient alike)",
     "NODE_WEIGHT = 0.1", "NODE_WEIGHT = 0.2"),
]


def _mlp_pins_fail(module):
    """Names of the scorer pins that fail with `module` in place of oracle.mlp."""
    import test_oracle_mlp as TM
    saved = TM.R
    TM.R = module
    failed = []
    try:
        checks = {"bf16": lambda: TM.test_bf16_rounding_by_hand(),
                  "layout": lambda: TM.test_param_count_and_layout(),
                  "finite differences": lambda: [TM.test_gradient_matches_finite_differences(w) for w in (1.0, 7.5)],
                  "forward": lambda: [TM.test_forward_by_hand(rb) for rb in (False, True)],
                  "loss": lambda: TM.test_loss_by_hand()}
        for name, fn in checks.items():
            try:
                fn()
            except (KeyboardInterrupt, SystemExit):
                raise
            except BaseException:
                failed.append(name)
    finally:
        TM.R = saved
    return failed


def _load_module(text, path):
    import importlib.util
    with open(path, "w") as f:
        f.write(text)
    spec = importlib.util.spec_from_file_location(os.path.splitext(os.path.basename(path))[0], path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_mlp_mutations_apply_once():
    src = open(MLP_SRC).read()
    for name, old, new in MLP_MUTANTS:
        assert src.count(old) == 1, name


def test_unmodified_scorer_reference_passes_its_pins(tmp_path):
    assert _mlp_pins_fail(_load_module(open(MLP_SRC).read(), str(tmp_path / "mlp_copy.py"))) == []


@pytest.mark.parametrize("k", range(len(MLP_MUTANTS)), ids=[m[0] for m in MLP_MUTANTS])
def test_each_planted_scorer_mistake_fails_a_pin(tmp_path, k):
    name, old, new = MLP_MUTANTS[k]
    mod = _load_module(open(MLP_SRC).read().replace(old, new), str(tmp_path / f"mlp_mutant{k}.py"))
    assert _mlp_pins_fail(mod), name


# --------------------------------------------------------------------------
# The solution set's plain definitions (oracle/definition.py): planted
# mistakes in copies of the module, each loaded in place of the original for
# the pins that use the definitions.

DEF_SRC = os.path.join(ROOT, "oracle", "definition.py")

DEF_MUTANTS = [
    ("binary vectors with the bit index off by one",
     "((idx[:, None] >> np.arange(k, dtype=np.int64)) & 1)",
     "((idx[:, None] >> (np.arange(k, dtype=np.int64) + 1)) & 1)"),
    ("meet in the middle joining A x2 + d instead of d - A x2",
     "S2 = d[None, :] - X2.astype(np.int64) @ A[:, h:].T",
     "S2 = d[None, :] + X2.astype(np.int64) @ A[:, h:].T"),
    ("solutions sorted by the last column first",
     "keys = [x[:, c] for c in range(n - 1, -1, -1)]", "keys = [x[:, c] for c in range(n)]"),
    ("box brute force without the upper bound",
     "    radix = r + 1\n", "    radix = r\n"),
]


def _def_pins_fail(module):
    """Names of the pins that fail with `module` in place of oracle.definition."""
    import test_oracle_bounds as TN
    import test_oracle_enum as TE
    saved = (TE.DEF, TN.DEF)
    TE.DEF = TN.DEF = module
    failed = []
    try:
        checks = {"hand example": lambda: TE.test_definition_hand_example(),
                  "methods agree": lambda: [TE.test_definition_methods_agree(s) for s in range(4)],
                  "enumeration": lambda: [TE.test_all_modes_equal_brute_force(TE.SMALL[k]) for k in range(3)],
                  "bounds": lambda: [TN.test_bounded_solution_sets_equal_brute_force(TN.CASES[k], 0, True)
                                     for k in range(3)]}
        for name, fn in checks.items():
            try:
                fn()
            except (KeyboardInterrupt, SystemExit):
                raise
            except BaseException:
                failed.append(name)
    finally:
        TE.DEF, TN.DEF = saved
    return failed


def test_definition_mutations_apply_once():
    src = open(DEF_SRC).read()
    for name, old, new in DEF_MUTANTS:
        assert src.count(old) == 1, name


def test_unmodified_definitions_pass_their_pins(tmp_path):
    assert _def_pins_fail(_load_module(open(DEF_SRC).read(), str(tmp_path / "definition_copy.py"))) == []


@pytest.mark.parametrize("k", range(len(DEF_MUTANTS)), ids=[m[0] for m in DEF_MUTANTS])
def test_each_planted_definition_mistake_fails_a_pin(tmp_path, k):
    name, old, new = DEF_MUTANTS[k]
    mod = _load_module(open(DEF_SRC).read().replace(old, new), str(tmp_path / f"definition_mutant{k}.py"))
    assert _def_pins_fail(mod), name
