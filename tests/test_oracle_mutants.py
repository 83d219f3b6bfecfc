"""Planted-mistake check of the oracle pins.

Each case copies oracle/pcr_oracle.c into a temporary directory, plants one
plausible mistake (a dropped term, a wrong sign, shift or index, a transposed
operand, a wrong tie-break), builds the copy and runs the pins of that part of
the oracle against it. Every planted mistake must make at least one pin fail. The oracle
in the tree is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pcr_oracle.c")

# (name, text in pcr_oracle.c, replacement); the first occurrence is replaced
MUTANTS = [
    ("eq1_no_min", "((double)v - (double)box_min)", "((double)v)"),
    ("eq1_scale", "floor(1073741824.0 *", "floor(2147483648.0 *"),
    ("words_reversed", "int shift = 20 - 10 * j;", "int shift = 10 * j;"),
    ("words_yz_swapped", "xs | (ys << 10) | (zs << 20)", "xs | (zs << 10) | (ys << 20)"),
    ("decode_shift", "v = (v << 10) |", "v = (v << 9) |"),
    ("morton_axis_order", "<< (3 * bit + a)", "<< (3 * bit + 2 - a)"),
    ("sort_unstable", "return x->idx < y->idx ? -1 : (x->idx > y->idx);",
     "return x->idx > y->idx ? -1 : (x->idx < y->idx);"),
    ("box_size_is_max", "B->size[a] = bmax[a] - bmin[a];", "B->size[a] = bmax[a];"),
    ("decode_no_min", "p[a] = b->min[a] + off;", "p[a] = off;"),
    ("decode_cell", "ldexpf(b->size[a], -10 * k)", "ldexpf(b->size[a], -10)"),
    ("project_transposed", "float cx = ((m[0] * x + m[4] * y) + m[8] * z) + m[12];",
     "float cx = ((m[0] * x + m[1] * y) + m[2] * z) + m[3];"),
    ("project_w_row", "float cw = ((m[3] * x + m[7] * y) + m[11] * z) + m[15];\n    if (!(cw > 0.0f)) return 0;",
     "float cw = ((m[2] * x + m[6] * y) + m[10] * z) + m[14];\n    if (!(cw > 0.0f)) return 0;"),
    ("pixel_no_offset", "(ndx * 0.5f + 0.5f)", "(ndx * 0.5f)"),
    ("pixel_y_flip", "(ndy * 0.5f + 0.5f)", "(0.5f - ndy * 0.5f)"),
    ("key_depth_from_x", "memcpy(&bits, &cw, 4);", "memcpy(&bits, &cx, 4);"),
    ("no_min_update", "if (key < vis[pix]) vis[pix] = key;", "vis[pix] = key;"),
    ("k_any_axis", "if (ex < T && ey < T) return 1;", "if (ex < T || ey < T) return 1;"),
    ("k2_threshold", "float T2 = T * 1024.0f;", "float T2 = T * 1000.0f;"),
    ("cull_any_corner", "if (row_max(sp, lo, hi) + mx < 0.0) return 1;",
     "if (row_min(sp, lo, hi) + mx < 0.0) return 1;"),
    ("cull_behind_any", "if (row_max(Wr, lo, hi) + g * bw <= 0.0) return 1;",
     "if (row_min(Wr, lo, hi) + g * bw <= 0.0) return 1;"),
    ("resolve_index", "color[(uint32_t)(vis[p] & 0xFFFFFFFFull)]", "color[(uint32_t)(vis[p] >> 32) & 3u]"),
    ("merge_max", "if (jobs[t].vis[p] < vis[p]) vis[p] = jobs[t].vis[p];",
     "if (jobs[t].vis[p] > vis[p] && jobs[t].vis[p] != OR_EMPTY) vis[p] = jobs[t].vis[p];"),
    ("index_not_global", "uint32_t i = b->first + j;\n            uint32_t pix;",
     "uint32_t i = j;\n            uint32_t pix;"),
    # per-frame counters (Table 2), their threaded merge, clamps, the culling
    # rounding bound, the resolve background, the view's rows and columns
    ("stats_points_k_one",
     "            st->points_k[k] += b->count;\n        }\n        for (uint32_t j = 0; j < b->count; ++j) {\n            uint32_t i = b->first + j;",
     "            st->points_k[k] += 1;\n        }\n        for (uint32_t j = 0; j < b->count; ++j) {\n            uint32_t i = b->first + j;"),
    ("stats_batches_k_fixed",
     "            st->batches_k[k] += 1;\n            st->points_k[k] += b->count;\n        }\n        for (uint32_t j = 0; j < b->count; ++j) {\n            uint32_t i = b->first + j;",
     "            st->batches_k[1] += 1;\n            st->points_k[k] += b->count;\n        }\n        for (uint32_t j = 0; j < b->count; ++j) {\n            uint32_t i = b->first + j;"),
    ("stats_accepted_all",
     "            if (!or_project_point(b, k, w1[i], w2[i], w3[i], i, v, &pix, &key)) continue;\n            if (st) st->points_accepted += 1;",
     "            if (st) st->points_accepted += 1;\n            if (!or_project_point(b, k, w1[i], w2[i], w3[i], i, v, &pix, &key)) continue;"),
    ("threaded_merge_drops_k", "                st->points_k[k] += jobs[t].st.points_k[k];",
     "                st->points_k[k] = jobs[t].st.points_k[k];"),
    ("threaded_merge_drops_batches", "            st->batches_rendered += jobs[t].st.batches_rendered;",
     "            st->batches_rendered = jobs[t].st.batches_rendered;"),
    ("morton_scale", "if (csize[a] > 0.0) t = floor(2097152.0 *", "if (csize[a] > 0.0) t = floor(1048576.0 *"),
    ("morton_no_clamp", "if (t > 2097151.0) t = 2097151.0;", ";"),
    ("eq1_no_clamp", "if (t > 1073741823.0) t = 1073741823.0;", ";"),
    ("cull_no_rounding_bound", "const double g = 6.0 * 0x1.0p-24;", "const double g = 0.0;"),
    ("cull_wide_margin", "const double e1 = 1.0 + 0x1.0p-10;", "const double e1 = 1.5;"),
    ("resolve_background", "out[p] = vis[p] == OR_EMPTY ? 0u : color",
     "out[p] = vis[p] == OR_EMPTY ? 0xFF000000u : color"),
    ("project_no_m12", "float cx = ((m[0] * x + m[4] * y) + m[8] * z) + m[12];",
     "float cx = ((m[0] * x + m[4] * y) + m[8] * z);"),
    ("pixel_width_for_y", "float fy = (ndy * 0.5f + 0.5f) * (float)v->height;",
     "float fy = (ndy * 0.5f + 0.5f) * (float)v->width;"),
    ("pixel_row_stride", "*pixel = py * v->width + px;", "*pixel = py * v->height + px;"),
    ("accept_right_edge", "if (!(fx >= 0.0f && fx < (float)v->width)) return 0;",
     "if (!(fx >= 0.0f && fx <= (float)v->width)) return 0;"),
    ("select_k_behind_1", "        if (!(cw > 0.0f)) return 3;\n        float f[2];",
     "        if (!(cw > 0.0f)) return 1;\n        float f[2];"),
    ("select_k_threshold_le", "if (ex < T && ey < T) return 1;", "if (ex <= T && ey <= T) return 1;"),
    ("decode_half_cell", "float off = fq * cell;", "float off = fq * cell * 0.5f;"),
    ("in_order_box_min_from_first",
     "                if (v < bmin[a]) bmin[a] = v;\n                if (v > bmax[a]) bmax[a] = v;\n            }\n        or_batch* B = &batches[b];\n        for (int a = 0; a < 3; ++a) {\n            B->min[a] = bmin[a];\n            B->size[a] = bmax[a] - bmin[a];\n        }\n        B->first = (uint32_t)first;",
     "                if (v > bmax[a]) bmax[a] = v;\n            }\n        or_batch* B = &batches[b];\n        for (int a = 0; a < 3; ++a) {\n            B->min[a] = bmin[a];\n            B->size[a] = bmax[a] - bmin[a];\n        }\n        B->first = (uint32_t)first;"),
]

# Sec. 3.6 high-quality shading, checked by the pins of tests/test_oracle_hqs.py
HQS_MUTANTS = [
    ("hqs_window_open", "if (!(w <= limit)) return;", "if (!(w < limit)) return;"),
    ("hqs_window_2pct", "float limit = wmin * 1.01f;", "float limit = wmin * 1.02f;"),
    ("hqs_window_none", "float limit = wmin * 1.01f;", "float limit = wmin;"),
    ("hqs_channel_shift", "sum[4 * (uint64_t)pix + 1] += (c >> 8) & 255u;",
     "sum[4 * (uint64_t)pix + 1] += (c >> 16) & 255u;"),
    ("hqs_no_count", "sum[4 * (uint64_t)pix + 3] += 1;", "sum[4 * (uint64_t)pix + 3] = 1;"),
    ("hqs_round_up", "(uint32_t)(sum[4 * p + 0] / n)", "(uint32_t)((sum[4 * p + 0] + n - 1) / n)"),
    ("hqs_lod_unselected", "if (!sel[i]) continue;\n        const or_batch* B = &nodes[i];\n        int k = or_select_k(B, v);\n        for",
     "const or_batch* B = &nodes[i];\n        int k = or_select_k(B, v);\n        for"),
    ("hqs_dilate_own_pixel", "best == OR_EMPTY ? 0u : hqs[at];",
     "best == OR_EMPTY ? 0u : hqs[(uint64_t)py * width + px];"),
    ("hqs_alpha_not_255", "((uint32_t)(sum[4 * p + 2] / n) << 16) | (255u << 24);",
     "((uint32_t)(sum[4 * p + 2] / n) << 16);"),
    ("hqs_blue_from_green", "sum[4 * (uint64_t)pix + 2] += (c >> 16) & 255u;",
     "sum[4 * (uint64_t)pix + 2] += (c >> 8) & 255u;"),
    ("hqs_red_plus_alpha", "sum[4 * (uint64_t)pix + 0] += c & 255u;",
     "sum[4 * (uint64_t)pix + 0] += (c & 255u) + (c >> 24);"),
    ("hqs_window_from_own_depth", "float limit = wmin * 1.01f;", "float limit = w * 1.01f;"),
    ("hqs_fixed_k3",
     "        int k = or_select_k(B, v);\n        for (uint32_t j = 0; j < B->count; ++j)\n"
     "            hqs_point(B, k, B->first + j, w1, w2, w3, color, v, vis, sum);\n    }\n"
     "    hqs_average(sum, npix, out);\n    free(sum);\n}",
     "        int k = 3;\n        for (uint32_t j = 0; j < B->count; ++j)\n"
     "            hqs_point(B, k, B->first + j, w1, w2, w3, color, v, vis, sum);\n    }\n"
     "    hqs_average(sum, npix, out);\n    free(sum);\n}"),
    ("hqs_lod_fixed_k3",
     "        const or_batch* B = &nodes[i];\n        int k = or_select_k(B, v);\n"
     "        for (uint32_t j = 0; j < B->count; ++j)\n            hqs_point",
     "        const or_batch* B = &nodes[i];\n        int k = 3;\n"
     "        for (uint32_t j = 0; j < B->count; ++j)\n            hqs_point"),
    ("hqs_threaded_drops_partials",
     "for (uint64_t q = 0; q < 4 * npix; ++q) jobs[0].sum[q] += jobs[t].sum[q];",
     "for (uint64_t q = 0; q < 4 * npix; ++q) jobs[0].sum[q] += 0;"),
    ("hqs_dilate_radius",
     "            int r = 1 + or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);\n"
     "            uint64_t best = OR_EMPTY, at = 0;",
     "            int r = or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);\n"
     "            uint64_t best = OR_EMPTY, at = 0;"),
    ("hqs_dilate_last_not_closest",
     "                    if (vis[q] < best) {\n                        best = vis[q];",
     "                    if (vis[q] != OR_EMPTY) {\n                        best = vis[q];"),
]

# the full-size encoding checker, checked by tests/test_oracle_verify.py
VERIFY_MUTANTS = [
    ("verify_no_order", "if (i > 0 && !(prev_code < code || (prev_code == code && prev_idx < idx))) {",
     "if (0) {"),
    ("verify_no_tiebreak", "(prev_code == code && prev_idx < idx)", "(prev_code == code)"),
    ("verify_no_box", "if (memcmp(&B->min[c], &bmin[c], 4) != 0 || memcmp(&B->size[c], &size, 4) != 0) {",
     "if (0) {"),
    ("verify_no_range", "if ((uint64_t)idx >= j->n) { j->code = 2; j->where = i; return NULL; }",
     "if (0) { j->code = 2; j->where = i; return NULL; }"),
    ("verify_lod_no_octant",
     "if (octant_of(p, &j->nodes[j->parent[c]]) != j->oct[c]) { j->code = 4; j->where = i; return NULL; }",
     ";"),
    ("verify_lod_no_priority", "if (any[b] && !pri_less(own_max[b], below[b])) { code = 5; *where = b; }",
     ";"),
    ("verify_lod_no_split_rule", "                         : (nodes[b].count > max_node_points && !last)) { code = 5; *where = b; }",
     "                         : 0) { code = 5; *where = b; }"),
    ("verify_lod_no_order", "(i > B->first && idx <= prev)", "(0)"),
    ("verify_no_header",
     "if (B->first != first || B->count != end - first) { j->code = 1; j->where = b; return NULL; }", ";"),
    ("verify_no_words",
     "            if (w[0] != j->w1[i] || w[1] != j->w2[i] || w[2] != j->w3[i]) {\n"
     "                j->code = 5; j->where = i; return NULL;\n            }", ""),
    ("verify_no_colour", "            if (col != j->color[i]) { j->code = 6; j->where = i; return NULL; }", ""),
    ("verify_batch_count",
     "if (batch_size == 0 || n > 0xFFFFFFFFull || nbatches != or_num_batches(n, batch_size)) return 1;",
     "if (batch_size == 0 || n > 0xFFFFFFFFull) return 1;"),
    ("verify_lod_no_words",
     "if (w[0] != j->w1[i] || w[1] != j->w2[i] || w[2] != j->w3[i]) { j->code = 6; j->where = i; return NULL; }",
     ";"),
    ("verify_lod_no_colour",
     "if ((j->rgba ? j->rgba[idx] : 0u) != j->color[i]) { j->code = 7; j->where = i; return NULL; }", ";"),
    ("verify_lod_no_root",
     "if (memcmp(&nodes[0].min[c], &lo[c], 4) != 0 || memcmp(&nodes[0].size[c], &side, 4) != 0) return 1;",
     ";"),
    ("verify_lod_no_header",
     "if (nodes[b].first != total || nodes[b].count == 0) { code = 1; *where = b; break; }", ";"),
    ("verify_lod_no_level",
     "if (p >= b || (b > 1 && p < parent[b - 1]) || level[b] != level[p] + 1 || level[b] >= max_levels) {",
     "if (p >= b || (b > 1 && p < parent[b - 1])) {"),
    ("verify_lod_no_child_cube",
     "            if (memcmp(&nodes[b].size[c], &half, 4) != 0) { code = 2; *where = b; }", ""),
    ("verify_lod_no_octant_order",
     "if (b > 1 && parent[b - 1] == p && oct[b - 1] >= o) { code = 2; *where = b; }", ";"),
    ("verify_lod_no_total", "if (!code && total != n) { code = 1; *where = nnodes; }", ";"),
]

# Sec. 3.5 level of detail and Sec. 3.7 foveation and dilation, checked by the
# pins of tests/test_oracle_lod.py
LOD_MUTANTS = [
    ("lod_root_not_cubic", "        if (e > side) side = e;\n    }\n    /* breadth-first",
     "        if (a == 0) side = e;\n    }\n    /* breadth-first"),
    ("lod_priority_seed", "pr[j].pri = or_splitmix64(((uint64_t)seed << 32) + w.idx[j]);",
     "pr[j].pri = or_splitmix64(((uint64_t)seed << 16) + w.idx[j]);"),
    ("lod_keep_largest", "if (x->pri != y->pri) return x->pri < y->pri ? -1 : 1;",
     "if (x->pri != y->pri) return x->pri > y->pri ? -1 : 1;"),
    ("lod_depth_limit", "if (w.n > max_node_points && w.level + 1 < max_levels) {",
     "if (w.n > max_node_points && w.level < max_levels) {"),
    ("lod_mid_quarter", "for (int a = 0; a < 3; ++a) mid[a] = w.lo[a] + half;",
     "for (int a = 0; a < 3; ++a) mid[a] = w.lo[a] + half * 0.5f;"),
    ("lod_child_corner", "for (int a = 0; a < 3; ++a) c->lo[a] = ((o >> a) & 1) ? mid[a] : w.lo[a];",
     "for (int a = 0; a < 3; ++a) c->lo[a] = ((o >> a) & 1) ? w.lo[a] + w.size : w.lo[a];"),
    ("lod_child_size", "c->size = half;", "c->size = w.size;"),
    ("lod_kept_priority_order", "qsort(kept, keep, sizeof(uint32_t), u32_cmp);   /* input order */",
     "/* kept in priority order */"),
    ("lod_select_no_parent", "if (ok && i > 0) ok = sel[parent[i]];", "if (0) ok = sel[parent[i]];"),
    ("lod_select_root_extent", "        int ok = !or_cull(&nodes[i], v);\n        if (ok && i > 0) {",
     "        int ok = !or_cull(&nodes[i], v);\n        if (ok) {"),
    ("lod_select_no_cull", "        int ok = !or_cull(&nodes[i], v);", "        int ok = 1;"),
    ("ring0_wider", "if (9.0f * d2 < r2) return 0;", "if (4.0f * d2 < r2) return 0;"),
    ("ring1_threshold", "if (ring == 1) t = (lod_px + lod_px_periphery) * 0.5f;",
     "if (ring == 1) t = lod_px;"),
    ("ring2_threshold", "if (ring == 2) t = lod_px_periphery;", "if (ring == 2) t = lod_px;"),
    ("dilate_radius",
     "            int r = 1 + or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);\n"
     "            uint64_t best = OR_EMPTY;",
     "            int r = or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);\n"
     "            uint64_t best = OR_EMPTY;"),
    ("dilate_ring_at_corner",
     "            int r = 1 + or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);\n"
     "            uint64_t best = OR_EMPTY;",
     "            int r = 1 + or_ring((float)px, (float)py, width, height);\n"
     "            uint64_t best = OR_EMPTY;"),
    ("dilate_farthest",
     "                    uint64_t k = vis[(uint64_t)y * width + (uint64_t)x];\n"
     "                    if (k < best) best = k;",
     "                    uint64_t k = vis[(uint64_t)y * width + (uint64_t)x];\n"
     "                    if (k != OR_EMPTY && (best == OR_EMPTY || k > best)) best = k;"),
]

CASES = ([m + ("test_oracle_pins.py",) for m in MUTANTS] +
         [m + ("test_oracle_hqs.py",) for m in HQS_MUTANTS] +
         [m + ("test_oracle_verify.py",) for m in VERIFY_MUTANTS] +
         [m + ("test_oracle_lod.py",) for m in LOD_MUTANTS])


@pytest.mark.parametrize("name,old,new,pins", CASES, ids=[m[0] for m in CASES])
def test_pins_catch_mutant(tmp_path, name, old, new, pins):
    with open(SRC) as f:
        src = f.read()
    assert old in src, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    cfile = tmp_path / "pcr_oracle.c"
    cfile.write_text(mutated)
    hdr = os.path.join(ROOT, "oracle", "pcr_oracle.h")
    (tmp_path / "pcr_oracle.h").write_text(open(hdr).read())
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", str(so), str(cfile), "-lm"])
    env = dict(os.environ, PCR_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"
