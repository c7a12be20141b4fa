"""The oracle's pins catch plausible mistakes: each case plants one mistake in a scratch copy of the
oracle (a dropped term, a wrong comparison, an off-by-one, a wrong tie rule), rebuilds it, and
expects the pin file that covers that function to fail.  Nothing is planted in the real oracle."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C, PY = "oracle/fq_oracle.c", "oracle/__init__.py"
CODEC, PX, BFS, PRED = ("tests/test_oracle_codec.py", "tests/test_oracle_px.py", "tests/test_oracle_bfs.py",
                        "tests/test_oracle_pred.py")

# (name, file, original text, planted text, occurrences, pin file expected to fail)
MUTATIONS = [
    ("width_one_bit_short", C, "    return bits;\n}", "    return bits > 1 ? bits - 1 : bits;\n}", 1, CODEC),
    ("encode_gap_without_minus_one", C, "uint64_t gap = (uint64_t)v[i] - (uint64_t)v[i - 1] - 1u;",
     "uint64_t gap = (uint64_t)v[i] - (uint64_t)v[i - 1];", 1, CODEC),
    ("decode_gap_without_plus_one", C, "            value = value + gap + 1u;\n            if (value > 0xFFFFFFFFu)",
     "            value = value + gap;\n            if (value > 0xFFFFFFFFu)", 1, CODEC),
    ("decode_without_block_order_check", C,
     "                    if (k > 0 && value <= out[i - 1u])\n                        return ORC_ECORRUPT;\n"
     "                    out[i] = (uint32_t)value;", "                    out[i] = (uint32_t)value;", 2, CODEC),
    ("packed_on_a_size_tie", C, "packed = (n > 0) && (packed_size < raw_size);",
     "packed = (n > 0) && (packed_size <= raw_size);", 3, CODEC),
    ("pad16_overshoots", C, "return (bytes + 15u) / 16u * 16u;", "return (bytes + 16u) / 16u * 16u;", 1, CODEC),
    ("bitmap_tie_to_clear", C, "mode = (2u * p <= nbits) ? ORC_FB_SET : ORC_FB_CLEAR;",
     "mode = (2u * p < nbits) ? ORC_FB_SET : ORC_FB_CLEAR;", 1, CODEC),
    ("bitmap_clear_decode_sets", C, "        else\n            words[q / 64u] &= ~((uint64_t)1u << (q % 64u));",
     "        else\n            words[q / 64u] |= ((uint64_t)1u << (q % 64u));", 1, CODEC),
    ("px_cost_tie_to_smaller_width", C, "if (cost <= best_cost) {", "if (cost < best_cost) {", 1, PX),
    ("px_exception_costs_4_bytes", C, "cost = 16u * b + 5u * e;", "cost = 16u * b + 4u * e;", 1, PX),
    ("fr_base_is_the_first_value", C, "if (v[i] < lo)\n                    lo = v[i];",
     "if (j == 0)\n                    lo = v[i];", 1, PRED),
    ("fr_width_one_bit_short", C, "        b[k] = (uint8_t)orc_bitlen((uint64_t)hi - lo);",
     "        b[k] = (uint8_t)(orc_bitlen((uint64_t)hi - lo) > 0 ? orc_bitlen((uint64_t)hi - lo) - 1 : 0);", 1, PRED),
    ("fr_decode_drops_the_base", C, "            out[i] = (uint32_t)(base + off);", "            out[i] = (uint32_t)(off);",
     1, PRED),
    ("parent_ranks_off_by_one", PY, "        out.append(r.astype(np.uint32))",
     "        out.append((r + (r + 1 < sets[d - 1].size)).astype(np.uint32))", 1, PRED),
    ("bfs_depth_plus_two", C, "depth[w] = depth[u] + 1;", "depth[w] = depth[u] + 2;", 1, BFS),
    ("validator_skips_adjacency", C, "        if (!found || depth[p] != depth[v] - 1)",
     "        if (depth[p] != depth[v] - 1)", 1, BFS),
    ("validator_allows_two_level_edges", C, "            if (a >= 0 && (a - c > 1 || c - a > 1))",
     "            if (a >= 0 && (a - c > 2 || c - a > 2))", 1, BFS),
    ("validator_skips_unreached_parents", C, "        if (depth[v] < 0 && parent[v] != 0xFFFFFFFFu)\n            return 4;",
     "        if (0)\n            return 4;", 1, BFS),
    ("bottom_up_count_skips_the_found_edge", C,
     "            total++;\n            if (depth[cols[e]] == d)\n                break;",
     "            if (depth[cols[e]] == d)\n                break;\n            total++;", 1, BFS),
    ("switch_to_bottom_up_on_equality", PY, "if direction == TOP_DOWN and m_f * alpha > m_u:",
     "if direction == TOP_DOWN and m_f * alpha >= m_u:", 1, BFS),
    ("switch_back_on_equality", PY, "elif direction == BOTTOM_UP and n_f * beta < n:",
     "elif direction == BOTTOM_UP and n_f * beta <= n:", 1, BFS),
    ("never_switch_back", PY, "elif direction == BOTTOM_UP and n_f * beta < n:", "elif False:", 1, BFS),
    ("bitmap_raw_only_when_strictly_larger", C, "    if (16u + inner_bytes >= raw_size) {",
     "    if (16u + inner_bytes > raw_size) {", 1, CODEC),
    ("raw_size_unpadded", C, "uint64_t orc_fq_raw_size(uint64_t n) { return 16u + pad16(4u * n); }",
     "uint64_t orc_fq_raw_size(uint64_t n) { return 16u + 4u * n; }", 1, CODEC),
    ("px_high_part_shifted_one_short", C, "            g[slot] |= high << bk;",
     "            g[slot] |= high << (bk ? bk - 1 : 0);", 1, PX),
    ("px_high_part_stored_unshifted", C, "put_u32(out + xhigh + 4u * x, (uint32_t)(gap >> b[k]));",
     "put_u32(out + xhigh + 4u * x, (uint32_t)(gap));", 1, PX),
    ("px_decode_accepts_zero_high_part", C, "            if (high == 0u || (high >> (32u - bk)) != 0u)",
     "            if ((high >> (32u - bk)) != 0u)", 1, PX),
    ("visited_stream_misses_its_own_level", PY,
     "            visited |= fbits\n            st, v = fb_encode(visited, n)",
     "            st, v = fb_encode(visited, n)\n            visited |= fbits", 1, BFS),
    ("container_counts_one_vertex_short", PY, "    reached = int(sum(f.size for f in sets))\n    head",
     "    reached = int(sum(f.size for f in sets)) - 1\n    head", 1, PRED),
    ("container_rank_streams_reversed", PY, "    for r in ranks:\n        st, q = fr_encode(r)",
     "    for r in ranks[::-1]:\n        st, q = fr_encode(r)", 1, PRED),
    ("m_u_counts_the_frontier", PY, "        visited_deg += m_f\n        m_u = total - visited_deg",
     "        m_u = total - visited_deg\n        visited_deg += m_f", 1, BFS),
]


@pytest.mark.parametrize("name,path,old,new,count,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, path, old, new, count, pins):
    for d in ("oracle", "tests", "paper_1704_00513_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__", "csrc", "test_oracle_mutations.py"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path)
    target = tmp_path / path
    text = target.read_text()
    assert text.count(old) == count, f"{name}: the planted site moved"
    target.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=600)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    # caught by a failing pin, not by a build or collection error
    assert r.returncode == 1 and " failed" in summary and "error" not in summary, \
        f"{name} was not caught:\n{r.stdout[-1500:]}{r.stderr[-1500:]}"
