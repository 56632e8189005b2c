"""Mutation check of the oracle's pins.

Each mutant below is a copy of one oracle source (``oracle/lv_oracle.c``,
``oracle/train_aux.py``, ``oracle/vertex.py`` or ``oracle/inplace.py``) with one plausible mistake
planted in it: a dropped term, a flipped sign, a swapped index or operand, an
off-by-one rank, a strict comparison made loose.  Every mutant is built on its
own (gcc for the C file; the numpy modules are loaded in place of the real
ones) and the oracle's pin tests (closed forms, invariants, brute force,
finite differences, hand traces; no GPU) are run against it in a child
process.  A mutant must make at least one pin fail; the unmodified
source, built the same way, must pass them all.  The mistakes are planted in
a temporary copy on the CPU; the oracle itself is never modified.

Every planted change keeps each memory access of the oracle in bounds, so a
mutant can only compute a wrong value.
"""
import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["tests/test_oracle_train.py", "tests/test_oracle_vertex.py", "tests/test_oracle_inplace.py",
             "tests/test_oracle_guards.py", "tests/test_oracle_adapt.py", "tests/test_oracle_render.py",
             "tests/test_oracle_segment.py"]

# (name, text in lv_oracle.c, replacement)
MUTANTS = [
    # rendering, Eq. 1-5
    ("alpha sign", "double alpha = -expm1(-sigma * l);", "double alpha = expm1(-sigma * l);"),
    ("T drops the chord", "T = T * exp(-sigma * l);", "T = T * exp(-sigma);"),
    ("trilinear x weight on the y bit", "double wx = (i & 1) ? u[0] : 1.0 - u[0];",
     "double wx = (i & 2) ? u[0] : 1.0 - u[0];"),
    ("density at chord entry", "local_coords(o, d, 0.5 * (t_in + t_out), g, u);\n  trilinear_weights(u, w8);",
     "local_coords(o, d, t_in, g, u);\n  trilinear_weights(u, w8);"),
    ("SH basis repeats a function", "Y[4] = c2a * x * y;", "Y[4] = c2a * x * z;"),
    ("SH degree-3 constant", "double c3d = sqrt(7.0 / (16.0 * pi));", "double c3d = sqrt(7.0 / (4.0 * pi));"),
    ("colour offset dropped", "raw[c] = s + 0.5;", "raw[c] = s;"),
    ("SH count of degree 3 is 10", "static int sh_count(int degree) { return (degree + 1) * (degree + 1); }",
     "static int sh_count(int degree) { return degree * degree + 1; }"),
    ("view direction reversed",
     "double d[3] = {(double)geom[4 * i] - cd->o[0], (double)geom[4 * i + 1] - cd->o[1],\n                   (double)geom[4 * i + 2] - cd->o[2]};",
     "double d[3] = {cd->o[0] - (double)geom[4 * i], cd->o[1] - (double)geom[4 * i + 1],\n                   cd->o[2] - (double)geom[4 * i + 2]};"),
    ("near-plane parameter taken as depth", "return c->z_near / dz;", "return c->z_near;"),
    ("candidates ordered by the near face", "    dkey[i] = f32_order_key(b.zc);\n", "    dkey[i] = f32_order_key(b.zc - g[3]);\n"),
    ("depth at chord entry", "*depth += w * tm;", "*depth += w * t_in;"),
    ("stop threshold halved", "if (T < t_stop) break;", "if (T < 0.5 * t_stop) break;"),
    ("w_max stores alpha", "wmax[id] = w;\n        warg[id] = gid;", "wmax[id] = alpha;\n        warg[id] = gid;"),
    ("w_max ties to the largest pixel", "(w == wmax[id] && (warg[id] < 0 || gid < warg[id]))",
     "(w == wmax[id] && (warg[id] < 0 || gid > warg[id]))"),
    ("chord not clipped at the near plane", "if (lo_t < t_near) { lo_t = t_near; din = 0.0; }",
     "if (lo_t < 0.0) { lo_t = 0.0; din = 0.0; }"),
    ("ray y through fx", "((double)y + 0.5 - c->cy) / c->fy", "((double)y + 0.5 - c->cy) / c->fx"),
    ("pixel corner instead of centre", "((double)x + 0.5 - c->cx) / c->fx", "((double)x - c->cx) / c->fx"),
    ("camera centre sign", "d->o[k] = -(d->R[0 * 3 + k] * d->t[0]", "d->o[k] = (d->R[0 * 3 + k] * d->t[0]"),
    ("exact segment: midpoint weight 2", "w8[i] = (wa[i] + 4.0 * w8[i] + wb[i]) / 6.0;",
     "w8[i] = (wa[i] + 2.0 * w8[i] + wb[i]) / 4.0;"),
    ("second view's pixels start one early", "    free_lists(&L);\n    pix_off += (int64_t)cd.W * cd.H;\n  }\n  if (w_max) {",
     "    free_lists(&L);\n    pix_off += (int64_t)cd.W * cd.H - 1;\n  }\n  if (w_max) {"),
    # backward
    ("backward: second view's pixels start one early",
     "    pix_off += (int64_t)cd.W * cd.H;\n  }\n  free(colors);\n  free(raw);",
     "    pix_off += (int64_t)cd.W * cd.H - 1;\n  }\n  free(colors);\n  free(raw);"),
    ("backward drops the later samples", "double ds = q->l * (Tk * a - S - Tf * gT);",
     "double ds = q->l * (Tk * a - Tf * gT);"),
    ("backward T-gradient sign", "double ds = q->l * (Tk * a - S - Tf * gT);",
     "double ds = q->l * (Tk * a - S + Tf * gT);"),
    ("backward uses T before the sample", "double ds = q->l * (Tk * a - S - Tf * gT);",
     "double ds = q->l * (q->T_before * a - S - Tf * gT);"),
    ("backward ignores the colour clamp", "if (!(raw[3 * i + ch] > 0.0)) continue;", "if (0) continue;"),
    ("backward ignores the density clamp", "if (q->sigma_raw > 0.0)\n", "if (1)\n"),
    ("backward depth term", "+ gD * q->t_mid;", "+ gD * q->l;"),
    # binning: pair list and statistics
    ("tile rect rounds the low edge up", "float a0 = floorf((umin - 1.0f) / fts)", "float a0 = ceilf((umin - 1.0f) / fts)"),
    ("tile index transposed", "uint64_t g = (uint64_t)(tile_off + (int64_t)ty * tiles_x + tx);",
     "uint64_t g = (uint64_t)(tile_off + (int64_t)tx * tiles_y + ty);"),
    ("equal pair keys ordered by the largest voxel id", "if (x->val != y->val) return x->val < y->val ? -1 : 1;\n  return 0;\n}\n\n/*\n * Sorted",
     "if (x->val != y->val) return x->val > y->val ? -1 : 1;\n  return 0;\n}\n\n/*\n * Sorted"),
    ("delta from the centre depth without the near clamp", "float dl = zs / c->fx;", "float dl = b.zc / c->fx;"),
    ("near-plane crossing parameter", "float f = (c->z_near - pz[i]) / dz;", "float f = (c->z_near - pz[j]) / dz;"),
    ("off-screen voxels marked seen", "      if (b.count == 0) continue;\n      float zs",
     "      if (b.culled) continue;\n      float zs"),
    ("depth key wrong for negative depths", "return (u & 0x80000000u) ? ~u : (u | 0x80000000u);",
     "return u | 0x80000000u;"),
    ("tile range end one short", "ranges[2 * g + 1] = (uint32_t)(q + 1);", "ranges[2 * g + 1] = (uint32_t)q;"),
    ("second view's tiles start one early", "tile_off += (int64_t)tiles_x * tiles_y;",
     "tile_off += (int64_t)tiles_x * tiles_y - 1;"),
    ("z_min from the last view", "if (zs < z_min[i]) z_min[i] = zs;", "if (1) z_min[i] = zs;"),
    ("delta_min from the last view", "if (dl < delta_min[i]) delta_min[i] = dl;", "if (1) delta_min[i] = dl;"),
    # pruning, Eq. 11-12 and guards i-iii
    ("EMA weights swapped", "float a = one_minus_alpha * m[i];\n    float c = alpha * x;",
     "float a = alpha * m[i];\n    float c = one_minus_alpha * x;"),
    ("hysteresis thresholds swapped", "if (mm < m_low) s[i] = 0;\n    else if (mm > m_high) s[i] = 1;",
     "if (mm < m_high) s[i] = 0;\n    else if (mm > m_low) s[i] = 1;"),
    ("hysteresis band open at m_low", "if (mm < m_low) s[i] = 0;", "if (mm <= m_low) s[i] = 0;"),
    ("hysteresis band open at m_high", "else if (mm > m_high) s[i] = 1;", "else if (mm >= m_high) s[i] = 1;"),
    ("quantile rank rounded down", "int64_t k = ppm_ceil(qb, cnt[b]);", "int64_t k = ppm_floor(qb, cnt[b]);"),
    ("inside score at the threshold", "w_max[i] > tau[bin[i]]", "w_max[i] >= tau[bin[i]]"),
    ("cap prunes the largest", "for (int64_t r = 0; r < cap; ++r) prune_mask[list[r].val] = 1;",
     "for (int64_t r = 0; r < cap; ++r) prune_mask[list[n_cand - 1 - r].val] = 1;"),
    ("cap counted over seen voxels", "int64_t cap = ppm_floor(cap_ppm, n);", "int64_t cap = ppm_floor(cap_ppm, ns);"),
    ("cap rounded up", "int64_t cap = ppm_floor(cap_ppm, n);", "int64_t cap = ppm_ceil(cap_ppm, n);"),
    ("depth bins reversed", "float num = z - p_lo;", "float num = p_hi - z;"),
    ("percentile rank rounded down", "int64_t k_lo = ppm_ceil(lo_ppm, m), k_hi = ppm_ceil(hi_ppm, m);",
     "int64_t k_lo = ppm_floor(lo_ppm, m), k_hi = ppm_floor(hi_ppm, m);"),
    ("keep-halo size test not strict", "prot |= h[4 * i + 3] < lim;", "prot |= h[4 * i + 3] <= lim;"),
    ("keep-halo edge test strict", "prot |= (w_max[i] >= halo_w && edge[i] >= halo_edge);",
     "prot |= (w_max[i] >= halo_w && edge[i] > halo_edge);"),
    ("q_b relaxes the far bins only", "if (dist < 0) dist = -dist;\n  int64_t den", "if (dist < 0) dist = 0;\n  int64_t den"),
    ("q_b bin centre off by one", "int64_t dist = 2 * (int64_t)b + 1 - n_bins;", "int64_t dist = 2 * (int64_t)b - n_bins;"),
    ("running percentile weights swapped", "float a0 = one_minus_r * state[0], b0 = r * *p_lo;",
     "float a0 = r * state[0], b0 = one_minus_r * *p_lo;"),
    ("running percentile returns the step's low value", "*p_lo = state[0];\n  *p_hi = state[1];\n}",
     "*p_lo = *p_lo;\n  *p_hi = state[1];\n}"),
    # subdivision, Eq. 13-16
    ("far bias sign", "float b = 1.0f + bz;", "float b = 1.0f - bz;"),
    ("eligibility not strict", "if (!(geom[4 * i + 3] > thr)) continue;", "if (!(geom[4 * i + 3] >= thr)) continue;"),
    ("level cap off by one", "if (!((int)level[i] < l_max)) continue;", "if (!((int)level[i] <= l_max)) continue;"),
    ("budget counts 8 per split", "int64_t kb = budget > n_alive ? (budget - n_alive) / 7 : 0;",
     "int64_t kb = budget > n_alive ? (budget - n_alive) / 8 : 0;"),
    ("top-k over all voxels", "int64_t k = ppm_floor(top_ppm, n_alive);", "int64_t k = ppm_floor(top_ppm, n);"),
    ("priority ties to the largest id", "return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);",
     "return x->id > y->id ? -1 : (x->id < y->id ? 1 : 0);"),
    ("child x offset flipped", "og[0] = g[0] + ((c & 1) ? hc : -hc);", "og[0] = g[0] + ((c & 1) ? -hc : hc);"),
    ("child corners copy the parent's", "q[1] = (float)(((c >> 1) & 1) + ((j >> 1) & 1)) * 0.5f;",
     "q[1] = (float)((j >> 1) & 1);"),
    ("child lerp order y before x", "float cy0 = lerp32(cx[0], cx[1], q[1]);", "float cy0 = lerp32(cx[0], cx[2], q[1]);"),
    ("child half size", "float hc = g[3] * 0.5f;", "float hc = g[3] * 0.25f;"),
    ("2-byte child fill dropped",
     "else if (aux_bytes[a] == 2) { uint16_t f = (uint16_t)aux_fill[a]; memcpy(dst, &f, 2); }",
     "else if (aux_bytes[a] == 2) { uint16_t f = 0; memcpy(dst, &f, 2); }"),
    ("survivor aux rows from the wrong voxel",
     "memcpy((char*)aux_out[a] + eb * (size_t)o, (const char*)aux_in[a] + eb * (size_t)i, eb);",
     "memcpy((char*)aux_out[a] + eb * (size_t)o, (const char*)aux_in[a] + eb * (size_t)o, eb);"),
    # LF-weighted loss, Eq. 7-10 and 18
    ("weight not inverted", "w[p] = pow(eps + 1.0 - s, gamma);", "w[p] = pow(eps + s, gamma);"),
    ("weight mean normalisation dropped", "double wt = w[p] / mean;", "double wt = w[p];"),
    ("Sobel y centre weight misplaced", "double gy = (YY(xm, yp) + 2.0 * YY(x, yp) + YY(xp, yp))",
     "double gy = (YY(xm, yp) + 2.0 * YY(xm, y) + YY(xp, yp))"),
    ("Sobel wraps the right border", "int xm = x > 0 ? x - 1 : 0, xp = x < W - 1 ? x + 1 : W - 1;",
     "int xm = x > 0 ? x - 1 : 0, xp = x < W - 1 ? x + 1 : 0;"),
    ("loss gradient factor", "dL_drgb[3 * (off + p) + c] = 2.0 / (3.0 * (double)np) * wt * r;",
     "dL_drgb[3 * (off + p) + c] = 1.0 / (3.0 * (double)np) * wt * r;"),
    ("edge percentile rank rounded down", "int64_t k = ppm_ceil(pctl_ppm, np);\n    if (k < 1) k = 1;\n    if (k > np)",
     "int64_t k = ppm_floor(pctl_ppm, np);\n    if (k < 1) k = 1;\n    if (k > np)"),
    ("luminance weights", "Y[p] = (G[3 * p] + G[3 * p + 1] + G[3 * p + 2]) / 3.0;",
     "Y[p] = (G[3 * p] + G[3 * p + 1] + G[3 * p + 1]) / 3.0;"),
    ("gamma ramp normalised by t1", "return gamma_max * (t - t0) / (t1 - t0);", "return gamma_max * (t - t0) / t1;"),
    ("Sobel wraps the bottom border", "int ym = y > 0 ? y - 1 : 0, yp = y < H - 1 ? y + 1 : H - 1;",
     "int ym = y > 0 ? y - 1 : 0, yp = y < H - 1 ? y + 1 : 0;"),
    ("loss gradient sign", "        double r = R[3 * p + c] - G[3 * p + c];", "        double r = G[3 * p + c] - R[3 * p + c];"),
    # a few more across the path
    ("z_min without the near clamp", "      float zs = fmaxf(b.zc, c->z_near);", "      float zs = b.zc;"),
    ("keep-halo ignored", "    if (s[i] == 0 && !prot) {", "    if (s[i] == 0) {"),
    ("trilinear z weight flipped", "double wz = (i & 4) ? u[2] : 1.0 - u[2];", "double wz = (i & 4) ? 1.0 - u[2] : u[2];"),
    ("backward colour gradient without the weight", "atomic_add(&dcol[3 * (int64_t)q->id + ch], w * gC[ch]);",
     "atomic_add(&dcol[3 * (int64_t)q->id + ch], gC[ch]);"),
]

# the numpy parts of the oracle: (name, file under oracle/, text, replacement)
PY_MUTANTS = [
    ("L_Tc gradient sign", "train_aux.py", "return loss, weight * (1.0 - 2.0 * T) / P",
     "return loss, weight * (2.0 * T - 1.0) / P"),
    ("L_Tc not averaged", "loss = weight * float(np.sum(T * (1.0 - T))) / P", "loss = weight * float(np.sum(T * (1.0 - T)))"),
    ("L_tv with face diagonals", "EDGES = [(c, c | b) for b in (1, 2, 4) for c in range(8) if not c & b]",
     "EDGES = [(c, c | b) for b in (1, 2, 3) for c in range(8) if not c & b]"),
    ("L_tv gradient sign at the second corner", "grad[:, j] -= 2.0 * diff", "grad[:, j] += 2.0 * diff"),
    ("Adam second moment corrected with beta1", "vhat = v / (1.0 - beta2 ** step)", "vhat = v / (1.0 - beta1 ** step)"),
    ("Adam eps inside the root", "(np.sqrt(vhat) + eps)", "np.sqrt(vhat + eps)"),
    ("Adam first moment rate", "m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g",
     "m = beta1 * np.asarray(m, np.float64) + (1.0 - beta2) * g"),
    ("L_tv gradient subtracted", "g = np.asarray(d_density, np.float64).reshape(-1, 8) + g_tv",
     "g = np.asarray(d_density, np.float64).reshape(-1, 8) - g_tv"),
    ("vertex ids ordered by x first", "vertex.py",
     "keys = q[..., 0] | (q[..., 1] << COORD_BITS) | (q[..., 2] << (2 * COORD_BITS))",
     "keys = q[..., 2] | (q[..., 1] << COORD_BITS) | (q[..., 0] << (2 * COORD_BITS))"),
    ("vertex key drops a coordinate", "vertex.py", "(q[..., 2] << (2 * COORD_BITS))", "(q[..., 2] << COORD_BITS)"),
    ("corner y bit read from z", "vertex.py", "1 if c & 2 else -1, 1 if c & 4", "1 if c & 4 else -1, 1 if c & 4"),
    ("tail rows move in decreasing order", "inplace.py", "move_from = np.flatnonzero(occupied[n_new:]) + n_new",
     "move_from = (np.flatnonzero(occupied[n_new:]) + n_new)[::-1]"),
    ("children appended before the holes fill", "inplace.py",
     "slots = np.concatenate([pruned[:min(h, others)], n + np.arange(max(0, others - h))])",
     "slots = np.concatenate([n + np.arange(max(0, others - h)), pruned[:min(h, others)]])"),
    ("child 0 not kept in the parent's row", "inplace.py", "child_dest[:, 0] = parents",
     "child_dest[:, 0] = parents[::-1]"),
    ("scatter overwrites", "vertex.py", "np.add.at(out, np.asarray(vidx).ravel(), np.asarray(corners, np.float64).ravel())",
     "out[np.asarray(vidx).ravel()] = np.asarray(corners, np.float64).ravel()"),
]
PY_MUTANTS = [m if len(m) == 4 else (m[0], "train_aux.py", m[1], m[2]) for m in PY_MUTANTS]

# pins that take seconds each run last, so that a mutant caught by a quick pin stops early
SLOW_PINS = ("test_pairs_cover_every_hit_pixel", "test_near_plane_straddler_tiles_cover_hits")

_RUNNER = r"""
import importlib.util
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import oracle
from oracle import oracle as O
O.build = lambda force=False: {lib!r}
O._lib = None
for mod_name, path in {py!r}.items():
    spec = importlib.util.spec_from_file_location("oracle." + mod_name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    sys.modules["oracle." + mod_name] = mod
    setattr(oracle, mod_name, mod)
import pytest

class SlowLast:
    def pytest_collection_modifyitems(self, items):
        items.sort(key=lambda it: any(s in it.nodeid for s in {slow!r}))

sys.exit(pytest.main({args!r}, plugins=[SlowLast()]))
"""


def _build(name, text, out_dir):
    path = os.path.join(out_dir, re.sub(r"\W+", "_", name) + ".so")
    src = path[:-3] + ".c"
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                    "-o", path, src, "-lm"], check=True, capture_output=True)
    return path


def _run_pins(lib_path, py_modules):
    """Return code of the pin tests against the C oracle at lib_path and the numpy modules py_modules
    ({name: path}), and the first failing test's id."""
    args = [os.path.join(ROOT, f) for f in PIN_FILES] + ["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                                                         "-rf", "--no-header", "-W", "ignore"]
    code = _RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib_path, py=py_modules, args=args,
                          slow=SLOW_PINS)
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    failed = re.findall(r"^FAILED (\S+)", r.stdout, flags=re.M)
    return r.returncode, (failed[0] if failed else None), r.stdout[-400:] + r.stderr[-400:]


def _planted(text, old, new, name):
    assert text.count(old) == 1, f"mutant {name!r}: its text occurs {text.count(old)} times"
    return text.replace(old, new)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    out_dir = str(tmp_path_factory.mktemp("oracle_mutants"))
    src = lambda f: open(os.path.join(ROOT, "oracle", f)).read()
    original = src("lv_oracle.c")
    jobs = {"(unmodified)": original}
    for name, old, new in MUTANTS:
        jobs[name] = _planted(original, old, new, name)
    with ThreadPoolExecutor(max_workers=8) as ex:
        libs = dict(zip(jobs, ex.map(lambda kv: _build(kv[0], kv[1], out_dir), jobs.items())))
    runs = {name: (lib, {}) for name, lib in libs.items()}
    for name, fname, old, new in PY_MUTANTS:
        path = os.path.join(out_dir, re.sub(r"\W+", "_", name) + ".py")
        with open(path, "w") as f:
            f.write(_planted(src(fname), old, new, name))
        runs[name] = (libs["(unmodified)"], {fname[:-3]: path})
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        return dict(zip(runs, ex.map(lambda r: _run_pins(*r), runs.values())))


def test_unmodified_oracle_passes_the_pins(outcomes):
    rc, _, tail = outcomes["(unmodified)"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS] + [m[0] for m in PY_MUTANTS])
def test_mutant_fails_a_pin(outcomes, name):
    rc, failed, tail = outcomes[name]
    # exit 1 with a failed pin named; a crash or an error before the pins ran counts for nothing
    assert rc == 1 and failed, f"mutant {name!r} survived the pins (exit {rc}): {tail}"
