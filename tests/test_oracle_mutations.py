"""The oracle's pins catch plausible mistakes: mutation tests on the CPU.

Each case copies oracle/oracle.c, plants one mistake (a wrong sign, a dropped
term, a transposed operand, an off-by-one, a wrong index or loop order), builds
the copy with gcc, and runs the oracle's pin suites against it through
MAXFLOW_ORACLE_LIB.  The suites are the step fixtures, the Dinic / closed-form /
brute-force / invariant pins, and the push-pull pins.  At least one pin must
fail.  A control build of the unmodified file must pass, which shows that the
copies are really the library under test.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
SUITES = ["tests/test_oracle_steps.py", "tests/test_oracle.py", "tests/test_oracle_pushpull.py"]

# (name, text in oracle.c (exactly one occurrence), replacement)
MUTANTS = [
    # 1. the current graph
    ("merge_overwrites_parallel_edges", "mc[out - 1] += E[i].c;", "mc[out - 1] = E[i].c;"),
    ("merge_keeps_self_loops", "if (src[i] == dst[i]) continue;", ""),
    # 2. Dinic
    ("dinic_no_reverse_credit", "g->res[path[i] ^ 1] += b;", "g->res[path[i] ^ 1] -= b;"),
    ("dinic_smax_forward_arcs", "if (g.res[b ^ 1] > 0 && !reach_t[x])", "if (g.res[b] > 0 && !reach_t[x])"),
    ("dinic_cut_dropped_negation", "if (smin[src[i]] && !smin[dst[i]]) c += cap[i];",
     "if (smin[src[i]] && smin[dst[i]]) c += cap[i];"),
    ("dinic_flow_wrong_arc", "(int32_t)(cap[i] - g.res[2 * i])", "(int32_t)(cap[i] - g.res[2 * i + 1])"),
    # 4. residual state
    ("rev_transposed", "r->rev[i] = rs_find(r, r->head[i], (int32_t)x);",
     "r->rev[i] = rs_find(r, (int32_t)x, r->head[i]);"),
    ("excess_sign", "e += r->cf[i] - r->cap[i];", "e += r->cap[i] - r->cf[i];"),
    ("set_flow_no_reverse_credit", "r->cf[r->rev[a]] += f[i];", "r->cf[r->rev[a]] -= f[i];"),
    ("static_init_dropped_term", "r->cf[j] = c_us + c_su;", "r->cf[j] = c_su;"),
    ("heights_forward_residual",
     "/* candidate predecessor z with edge (z, y) */\n"
     "            if (z != s && r->h[z] == n && r->cf[r->rev[i]] > 0) {",
     "/* candidate predecessor z with edge (z, y) */\n            if (z != s && r->h[z] == n && r->cf[i] > 0) {"),
    ("heights_step_two",
     "r->cf[r->rev[i]] > 0) {\n                r->h[z] = r->h[y] + 1;\n"
     "                queue[tail++] = z;\n            }\n        }\n    }\n    free(queue);\n    if (h_out)",
     "r->cf[r->rev[i]] > 0) {\n                r->h[z] = r->h[y] + 2;\n"
     "                queue[tail++] = z;\n            }\n        }\n    }\n    free(queue);\n    if (h_out)"),
    ("heights_no_deficit_roots", "if (deficit_roots)\n", "if (0)\n"),
    ("heights_label_the_source",
     "/* candidate predecessor z with edge (z, y) */\n"
     "            if (z != s && r->h[z] == n && r->cf[r->rev[i]] > 0) {",
     "/* candidate predecessor z with edge (z, y) */\n            if (r->h[z] == n && r->cf[r->rev[i]] > 0) {"),
    ("apply_capacity_sign", "r->cf[a] += U[i].c - r->cap[a];", "r->cf[a] += r->cap[a] - U[i].c;"),
    ("apply_clamp_sign", "r->cf[r->rev[i]] += r->cf[i];", "r->cf[r->rev[i]] -= r->cf[i];"),
    ("apply_source_step_dropped_term", "r->e[u] += d;\n            r->e[s] -= d;\n",
     "r->e[u] += d;\n"),
    ("apply_first_update_wins", "for (i = B - 1; i >= 0; i--) {", "for (i = 0; i < B; i++) {"),
    ("apply_insertion_resets_carried_flow",
     "r2->cf[rs_find(r2, (int32_t)x, r->head[j])] = r->cf[j];",
     "r2->cf[rs_find(r2, (int32_t)x, r->head[j])] = r->cap[j];"),
    ("slots_placeholder_counted_as_capacity",
     "if (S[i].c >= 0) S[K - 1].c = (S[K - 1].c < 0 ? 0 : S[K - 1].c) + S[i].c;",
     "if (S[i].c >= 0) S[K - 1].c = S[K - 1].c + S[i].c;"),
    ("certificate_cut_counts_inner_edges",
     "if (r->h[r->head[i]] == r->n) continue;\n            c += r->cap[i];",
     "c += r->cap[i];"),
    ("value_counts_source_side", "if (x != s && r->h[x] < r->n) v += r->e[x];",
     "if (x != s && r->h[x] <= r->n) v += r->e[x];"),
    ("value_drops_deficits", "if (x != s && r->h[x] < r->n) v += r->e[x];",
     "if (x != s && r->h[x] < r->n && r->e[x] > 0) v += r->e[x];"),
    # Alg. 2 / Alg. 3
    ("discharge_tie_to_last_slot",
     "if (r->cf[j] > 0 && r->h[r->head[j]] < hbest) { best = j; hbest = r->h[r->head[j]]; }",
     "if (r->cf[j] > 0 && r->h[r->head[j]] <= hbest) { best = j; hbest = r->h[r->head[j]]; }"),
    ("discharge_relabel_without_plus_one",
     "r->h[u] = (best < 0 || hbest >= n - 1) ? n : hbest + 1;\n            if (relabels)",
     "r->h[u] = (best < 0 || hbest >= n - 1) ? n : hbest;\n            if (relabels)"),
    ("discharge_relabel_not_clamped",
     "r->h[u] = (best < 0 || hbest >= n - 1) ? n : hbest + 1;\n            if (relabels)",
     "r->h[u] = (best < 0) ? n : hbest + 1;\n            if (relabels)"),
    ("discharge_push_ignores_excess", "int64_t d = min64(r->e[u], r->cf[best]);", "int64_t d = r->cf[best];"),
    ("discharge_no_reverse_credit", "r->cf[r->rev[best]] += d;", "r->cf[r->rev[best]] -= d;"),
    ("discharge_runs_when_inactive", "if (!(r->h[u] < n && r->e[u] > 0)) continue;",
     "if (!(r->h[u] <= n && r->e[u] > 0)) continue;"),
    ("remove_invalid_off_by_one", "if (r->cf[j] > 0 && r->h[x] > r->h[v] + 1) {",
     "if (r->cf[j] > 0 && r->h[x] > r->h[v] + 2) {"),
    ("remove_invalid_wrong_index", "r->e[x] -= c;\n                r->e[v] += c;",
     "r->e[x] -= c;\n                r->e[x] += c;"),
    # 5. Sec. 5.2.2 push and pull
    ("saturate_sink_sign", "r->e[z] -= d;\n            r->e[t] += d;", "r->e[z] += d;\n            r->e[t] += d;"),
    ("pull_heights_backward_residual", "if (z != t && r->h[z] == n && r->cf[i] > 0) {",
     "if (z != t && r->h[z] == n && r->cf[r->rev[i]] > 0) {"),
    ("pull_heights_label_the_sink", "if (z != t && r->h[z] == n && r->cf[i] > 0) {",
     "if (r->h[z] == n && r->cf[i] > 0) {"),
    ("push_side_roots_from_the_other_side",
     "if (x != s && x != t && r->e[x] < 0 && (!side || side[x] == want)) { r->h[x] = 0; queue[tail++] = x; }",
     "if (x != s && x != t && r->e[x] < 0 && (!side || side[x] != want)) { r->h[x] = 0; queue[tail++] = x; }"),
    ("pull_roots_from_the_other_side",
     "if (x != s && x != t && r->e[x] > 0 && (!side || side[x] == want)) { r->h[x] = 0; queue[tail++] = x; }",
     "if (x != s && x != t && r->e[x] > 0 && (!side || side[x] != want)) { r->h[x] = 0; queue[tail++] = x; }"),
    ("pull_value_sign", "v -= r->e[x];", "v += r->e[x];"),
    ("pull_discharge_ignores_deficit", "int64_t d = min64(-r->e[u], r->cf[in]);", "int64_t d = r->cf[in];"),
    ("pull_remove_invalid_off_by_one", "if (r->cf[in] > 0 && r->h[x] > r->h[z] + 1) {",
     "if (r->cf[in] > 0 && r->h[x] > r->h[z] + 2) {"),
    ("saturate_cut_wrong_side", "if (side[v] == 1 && d > 0) {", "if (side[v] == 0 && d > 0) {"),
    ("cut_side_inverted", "side[x] = r->h[x] < r->n ? 1 : 0;", "side[x] = r->h[x] < r->n ? 0 : 1;"),
]


def _build(tmp_path, text, tag):
    c = tmp_path / f"oracle_{tag}.c"
    so = tmp_path / f"liboracle_{tag}.so"
    c.write_text(text)
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", str(c), "-o", str(so)])
    return str(so)


def _run_pins(lib, timeout=240):
    env = dict(os.environ, MAXFLOW_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *SUITES]
    try:
        r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return None, "timed out"
    return r.returncode, r.stdout[-2000:]


def test_control_copy_passes_and_is_the_library_used(tmp_path):
    lib = _build(tmp_path, open(SRC).read(), "control")
    env = dict(os.environ, MAXFLOW_ORACLE_LIB=lib)
    out = subprocess.run([sys.executable, "-c", "import oracle; oracle.maxflow(2, [0], [1], [1], 0, 1); "
                          "import oracle as o; print(o.library_path())"],
                         cwd=ROOT, env=env, capture_output=True, text=True, check=True).stdout.split()[-1]
    assert out == lib
    rc, tail = _run_pins(lib)
    assert rc == 0, tail


@pytest.mark.parametrize("name,find,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_a_planted_mistake_fails_a_pin(tmp_path, name, find, repl):
    text = open(SRC).read()
    assert text.count(find) == 1, f"{name}: the mutation site must occur exactly once"
    lib = _build(tmp_path, text.replace(find, repl), name)
    rc, tail = _run_pins(lib)
    assert rc != 0, f"{name} survived every pin:\n{tail}"


# The scheduler network's numpy reference (oracle/mlp_ref.py), pinned by
# tests/test_mlp_ref.py: finite differences, torch autograd, torch's Adam.
MLP_SRC = os.path.join(ROOT, "oracle", "mlp_ref.py")
MLP_MUTANTS = [
    ("forward_drops_a_bias", "a2 = h1 @ W2.T + b2", "a2 = h1 @ W2.T"),
    ("forward_without_relu", "h1 = np.maximum(a1, 0.0)", "h1 = a1"),
    ("loss_mean_over_all_outputs", "return float((m * d * d).sum() / m.sum())",
     "return float((m * d * d).sum() / m.size)"),
    ("grad_ignores_the_mask", "dy = 2.0 * m * (y - np.asarray(t, np.float64).reshape(y.shape)) / m.sum()",
     "dy = 2.0 * (y - np.asarray(t, np.float64).reshape(y.shape)) / m.sum()"),
    ("grad_wrong_relu_gate", "dh2 = (dy @ W3) * (a2 > 0)", "dh2 = (dy @ W3) * (a2 >= 0) * (a1 > 0)"),
    ("grad_drops_bias_term", "gb2 = dh2.sum(0)", "gb2 = 0.0 * dh2.sum(0)"),
    ("layout_biases_first", "for shape in ((H, n_in), (H,), (H, H), (H,), (n_out, H), (n_out,)):",
     "for shape in ((H,), (H, n_in), (H, H), (H,), (n_out, H), (n_out,)):"),
    ("adam_first_moment_of_squares", "m2 = b2 * m2 + (1 - b2) * g * g", "m2 = b2 * m2 + (1 - b2) * g * abs(g)"),
    ("adam_no_bias_correction", "mh = m1 / (1 - b1 ** step)", "mh = m1"),
    ("adam_eps_inside_sqrt", "np.sqrt(vh) + eps", "np.sqrt(vh + eps)"),
]

_MLP_DRIVER = """
import importlib.util, sys
import oracle
spec = importlib.util.spec_from_file_location("oracle.mlp_ref", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
sys.modules["oracle.mlp_ref"] = mod
oracle.mlp_ref = mod
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "tests/test_mlp_ref.py"]))
"""


def _run_mlp_pins(path):
    r = subprocess.run([sys.executable, "-c", _MLP_DRIVER, path], cwd=ROOT, capture_output=True, text=True,
                       timeout=240)
    return r.returncode, r.stdout[-2000:]


def test_mlp_control_copy_passes(tmp_path):
    f = tmp_path / "mlp_ref_control.py"
    f.write_text(open(MLP_SRC).read())
    rc, tail = _run_mlp_pins(str(f))
    assert rc == 0, tail


@pytest.mark.parametrize("name,find,repl", MLP_MUTANTS, ids=[m[0] for m in MLP_MUTANTS])
def test_a_planted_mistake_in_the_network_reference_fails_a_pin(tmp_path, name, find, repl):
    text = open(MLP_SRC).read()
    assert text.count(find) == 1, f"{name}: the mutation site must occur exactly once"
    f = tmp_path / f"mlp_ref_{name}.py"
    f.write_text(text.replace(find, repl))
    rc, tail = _run_mlp_pins(str(f))
    assert rc != 0, f"{name} survived every pin:\n{tail}"
