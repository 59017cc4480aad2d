"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them.  The mistakes are planted on the CPU, in a
temporary copy of serialwt.c; the committed oracle is never modified."""
import json
import os

import numpy as np
import pytest

from paper_1407_8142_gb300 import synth
from tests.test_oracle_pins import n_levels, sortwt_levels, unpack, walk_access

HERE = os.path.dirname(os.path.abspath(__file__))

# (name, original text, planted text, occurrences replaced)
MUTANTS = [
    ("dropped X_s term", "nxt[start + xs + rights] = s;", "nxt[start + rights] = s;"),
    ("bit index from the bottom", "const uint32_t mask = 1u << (L - (l + 1));",
     "const uint32_t mask = 1u << l;"),
    ("off-by-one level bit", "const uint32_t mask = 1u << (L - (l + 1));",
     "const uint32_t mask = 1u << (L - l - (l > 0 ? 2 : 1));"),
    ("inclusive directory", "if ((i & 511) == 0) D[i >> 9] = ones;\n      ones += (B[i >> 5] >> (i & 31)) & 1u;",
     "ones += (B[i >> 5] >> (i & 31)) & 1u;\n      if ((i & 511) == 0) D[i >> 9] = ones;"),
    ("swapped child ids", "A2[na2].id = 2 * id + 1;", "A2[na2].id = 2 * id + 3;"),
    ("unstable left child", "nxt[start + lefts] = s;", "nxt[start + xs - 1 - lefts] = s;"),
    ("MSB-first words", "1u << ((start + i) & 31);", "1u << (31 - ((start + i) & 31));"),
    ("zeros count", "zeros[l] = n - ones;", "zeros[l] = ones;"),
    ("exclusive rank query", "for (uint64_t j = 0; j <= idx[q]; ++j)", "for (uint64_t j = 0; j < idx[q]; ++j)"),
    ("select off by one", "if (sym_at(S, j, b) == c[q] && ++seen == k[q])",
     "if (sym_at(S, j, b) == c[q] && seen++ == k[q])"),
    ("early stop one level too soon", "if (r <= 2) {", "if (r <= 4) {"),
    ("right child start", "A2[na2].start = start + xs;", "A2[na2].start = start + xs - 1;"),
    ("access returns neighbour", "out[q] = idx[q] < n ? sym_at(S, idx[q], b) : UINT32_MAX;",
     "out[q] = idx[q] + 1 < n ? sym_at(S, idx[q] + 1, b) : UINT32_MAX;"),
]


def pins_pass(o, lib) -> bool:
    """Run a compact version of every pin against the bound library."""
    try:
        with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
            for e in json.load(f)["examples"]:
                S = np.array(e["S"], dtype=np.uint8)
                res = o.build(S, e["sigma"], lib=lib)
                if res["bits"][:, 0].tolist() != e["word0"]:
                    return False
                if res["rank"].tolist() != e["rank"] or res["zeros"].tolist() != e["zeros"]:
                    return False
                nodes = [[int(a), int(b), int(c)] for a, b, c in
                         zip(res["node_id"], res["node_start"], res["node_len"])]
                if nodes != e["nodes"]:
                    return False
        with open(os.path.join(HERE, "golden", "query_examples.json")) as f:
            for e in json.load(f)["examples"]:
                S = np.array(e["S"], dtype=np.uint8)
                a, r, q = e["access"], e["rank"], e["select"]
                got = o.access(S, np.array(a["i"], dtype=np.uint64), lib=lib)
                if [int(x) if int(x) != 2**32 - 1 else -1 for x in got] != a["out"]:
                    return False
                got = o.rank(S, e["sigma"], np.array(r["c"]), np.array(r["i"]), lib=lib)
                if [int(x) for x in got] != r["out"]:
                    return False
                got = o.select(S, e["sigma"], np.array(q["c"]), np.array(q["k"]), lib=lib)
                if [int(x) if int(x) != 2**64 - 1 else -1 for x in got] != q["out"]:
                    return False
        for sigma, b, n in ((256, 1, 1500), (5, 1, 100), (3000, 2, 700)):
            S = synth.zipf(n, sigma, 1.0, b, 7)
            res = o.build(S, sigma, lib=lib)
            ref = sortwt_levels(S, sigma)
            levels = [unpack(res["bits"][l], n) for l in range(res["L"])]
            for l in range(n_levels(sigma)):
                if levels[l].tolist() != ref[l]:
                    return False
                cum = np.concatenate([[0], np.cumsum(levels[l])])
                D = [int(cum[min(512 * k, n)]) for k in range((n + 511) // 512 + 1)]
                if res["rank"][l].tolist() != D:
                    return False
            if [walk_access(levels, n, i) for i in range(0, n, 5)] != S[::5].astype(np.int64).tolist():
                return False
            idx = np.arange(0, n, 3, dtype=np.uint64)
            if o.access(S, idx, lib=lib).tolist() != S[::3].tolist():
                return False
            c = S[::3].astype(np.uint32)
            r = o.rank(S, sigma, c, idx, lib=lib)
            want = [int(np.count_nonzero(S[: int(i) + 1] == x)) for i, x in zip(idx, c)]
            if r.tolist() != want:
                return False
            if o.select(S, sigma, c, r, lib=lib).tolist() != idx.tolist():
                return False
    except Exception:
        return False
    return True


def test_original_passes(oracle_mod, tmp_path):
    lib = oracle_mod.compile_variant(oracle_mod.source_text(), str(tmp_path / "orig"))
    assert pins_pass(oracle_mod, lib)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name, old, new):
    src = oracle_mod.source_text()
    assert old in src, f"mutation site for '{name}' not found"
    lib = oracle_mod.compile_variant(src.replace(old, new), str(tmp_path / "m"))
    assert not pins_pass(oracle_mod, lib), f"planted mistake '{name}' was not caught"


# Mistakes planted in the wavelet-matrix builder (Section 7); each site is
# unique to it.
MATRIX_MUTANTS = [
    ("ones before zeros",
     "if (cur[i] & mask) nxt[z + rights++] = cur[i];\n      else nxt[lefts++] = cur[i];",
     "if (cur[i] & mask) nxt[rights++] = cur[i];\n      else nxt[(n - z) + lefts++] = cur[i];"),
    ("unstable ones", "if (cur[i] & mask) nxt[z + rights++] = cur[i];",
     "if (cur[i] & mask) nxt[n - 1 - rights++] = cur[i];"),
    ("unstable zeros", "else nxt[lefts++] = cur[i];", "else nxt[z - 1 - lefts++] = cur[i];"),
    ("no reordering between levels",
     "    uint32_t *t = cur; cur = nxt; nxt = t;\n  }\n  wto_directory(bits, n, L, rank, zeros);\n  free(cur); free(nxt);\n",
     "  }\n  wto_directory(bits, n, L, rank, zeros);\n  free(cur); free(nxt);\n"),
    ("bit index from the bottom",
     "const uint32_t mask = 1u << (L - (l + 1));\n    uint32_t *B = bits + (uint64_t)l * W;\n    uint64_t z = 0;",
     "const uint32_t mask = 1u << l;\n    uint32_t *B = bits + (uint64_t)l * W;\n    uint64_t z = 0;"),
]


def matrix_pins_pass(o, lib) -> bool:
    from tests.test_oracle_matrix_pins import mx_access, sorted_levels
    try:
        with open(os.path.join(HERE, "golden", "matrix_examples.json")) as f:
            for e in json.load(f)["examples"]:
                res = o.matrix_build(np.array(e["S"], dtype=np.uint8), e["sigma"], lib=lib)
                if res["bits"][:, 0].tolist() != e["word0"] or res["zeros"].tolist() != e["zeros"]:
                    return False
                if res["rank"].tolist() != e["rank"]:
                    return False
        for sigma, b, n in ((256, 1, 1200), (11, 1, 300), (70000, 4, 500)):
            S = synth.zipf(n, sigma, 1.0, b, 5)
            res = o.matrix_build(S, sigma, lib=lib)
            levels = [unpack(res["bits"][l], n).astype(np.int64) for l in range(res["L"])]
            ref = sorted_levels(S, sigma)
            if [lv.tolist() for lv in levels] != ref:
                return False
            zeros = [int(z) for z in res["zeros"]]
            if [mx_access(levels, zeros, i) for i in range(0, n, 7)] != S[::7].astype(np.int64).tolist():
                return False
    except Exception:
        return False
    return True


def test_matrix_original_passes(oracle_mod, tmp_path):
    lib = oracle_mod.compile_variant(oracle_mod.source_text(), str(tmp_path / "orig"))
    assert matrix_pins_pass(oracle_mod, lib)


@pytest.mark.parametrize("name,old,new", MATRIX_MUTANTS, ids=[m[0] for m in MATRIX_MUTANTS])
def test_matrix_planted_mistake_is_caught(oracle_mod, tmp_path, name, old, new):
    src = oracle_mod.source_text()
    assert src.count(old) == 1, f"mutation site for '{name}' not unique"
    lib = oracle_mod.compile_variant(src.replace(old, new), str(tmp_path / "m"))
    assert not matrix_pins_pass(oracle_mod, lib), f"planted mistake '{name}' was not caught"
