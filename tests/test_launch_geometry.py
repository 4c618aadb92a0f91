"""Launch geometry and index maps of the CUDA kernels, checked on the CPU.

compute-sanitizer is not available to these tests, so the index arithmetic of
the two largest kernels is restated here and checked against the buffers it
addresses and against the oracle's own numbering:

* patch smoother (Algorithm 2): which lines each thread of a pass transforms,
  which patch a CTA takes in each of the three
  launch kinds (every patch / interior patches / boundary patches), and the
  global DoF of every patch-local unknown.  The restated map must give the
  oracle's patch DoF set R_j in the same order, stay inside the vector, touch
  no constrained boundary-normal DoF, and give disjoint sets to the patches of
  one colour (the scatter x += R_j^T (U, P) has no atomics).
* operator apply: the persistent CTAs' equal shares of all columns' cells,
  numbered block row by block row and marched as runs inside blocks, write
  every velocity entry exactly once, and the 32-bit per-CTA staging offsets
  fit for every mesh the library accepts.
* level transfers: the prolongation's plain += reaches every free fine node
  exactly once, and the restriction's atomic adds reach each coarse node at
  most twice (two adds onto zero give the same sum in either order).
"""
import numpy as np
import pytest

from oracle.discretization import Discretization
from oracle.multigrid import colour_vertices, patch_dofs

# ---------------------------------------------------------------- patch kernel
# Restated from the library: colour_counts, interior_box (smoother.cu), the
# blk -> vertex decode and patch_node_global / patch_local_decode
# (patch_kernel.cuh).


def colour_counts(n, colour):
    return [n // 2 if (colour >> d) & 1 else (n - 1) // 2 for d in range(3)]


def interior_box(n, colour, cnt):
    tlo, cint = [], []
    for d in range(3):
        bit = (colour >> d) & 1
        lo, hi = cnt[d], 0
        for t in range(cnt[d]):
            v = 2 * t + 1 if bit else 2 * t + 2
            if 2 <= v <= n - 2:
                lo, hi = min(lo, t), max(hi, t + 1)
        tlo.append(lo)
        cint.append(max(0, hi - lo))
    return tlo, cint


def patch_of_block(blk, n, colour, part, cnt, tlo, cint):
    """Vertex of CTA blk, or None where the boundary launch skips the patch."""
    p, v = blk, []
    for d in range(3):
        ext = cint[d] if part == 1 else cnt[d]
        t = (tlo[d] if part == 1 else 0) + p % ext
        p //= ext
        v.append(2 * t + 1 if (colour >> d) & 1 else 2 * t + 2)
    interior = all(2 <= v[d] <= n - 2 for d in range(3))
    if part == 2 and interior:
        return None
    return tuple(v)


def patch_local_decode(j, k):
    npc, npd = 2 * k + 1, 2 * k + 2
    nv1 = npc * npd * npd
    if j < 3 * nv1:
        c = j // nv1
        li = j - c * nv1
        e0 = npc if c == 0 else npd
        e1 = npc if c == 1 else npd
        return c, li % e0, (li // e0) % e1, li // (e0 * e1)
    q = j - 3 * nv1
    return 3, q % npd, (q // npd) % npd, q // (npd * npd)


def patch_node_global(c, i, v, k, m):
    nd = k + 1
    nvel = (m + 1) * m * m
    g = [(v[d] - 1) * nd + i[d] + (1 if d == c else 0) for d in range(3)]
    if c < 3:
        e0 = m + 1 if c == 0 else m
        e1 = m + 1 if c == 1 else m
        return c * nvel + g[0] + e0 * (g[1] + e1 * g[2])
    return 3 * nvel + g[0] + m * (g[1] + m * g[2])


def patch_map(v, k, m):
    npc, npd = 2 * k + 1, 2 * k + 2
    nl = 3 * npc * npd * npd + npd ** 3
    out = np.empty(nl, dtype=np.int64)
    for j in range(nl):
        c, i0, i1, i2 = patch_local_decode(j, k)
        out[j] = patch_node_global(c, (i0, i1, i2), v, k, m)
    return out


@pytest.mark.parametrize("n,k", [(2, 1), (3, 2), (4, 1), (5, 3), (6, 2), (7, 1), (8, 2), (4, 5), (9, 1)])
def test_patch_index_map_equals_the_oracle_patch_sets(n, k):
    d = Discretization(n, k)
    free = d.free_mask()
    for colour in range(8):
        cnt = colour_counts(n, colour)
        tlo, cint = interior_box(n, colour, cnt)
        every = [patch_of_block(b, n, colour, 0, cnt, tlo, cint) for b in range(int(np.prod(cnt)))]
        inner = [patch_of_block(b, n, colour, 1, cnt, tlo, cint) for b in range(int(np.prod(cint)))]
        outer = [patch_of_block(b, n, colour, 2, cnt, tlo, cint) for b in range(int(np.prod(cnt)))]
        outer = [v for v in outer if v is not None]
        expect = sorted(colour_vertices(n, colour))
        assert sorted(every) == expect
        # the split launches take every patch exactly once
        assert sorted(inner + outer) == expect
        assert all(2 <= v[e] <= n - 2 for v in inner for e in range(3))
        seen = np.zeros(d.N, dtype=np.int32)
        for v in every:
            g = patch_map(v, k, d.m)
            assert np.array_equal(g, patch_dofs(d, v)), (colour, v)
            assert g.min() >= 0 and g.max() < d.N
            assert free[g].all()
            seen[g] += 1
        assert seen.max() <= 1, f"patches of colour {colour} share a DoF"


# Restated from PatchThreads and patch_pass (patch_kernel.cuh): W warps per
# velocity component (FP32: 1 for k <= 2, 2 for k = 3, 4, 3 for k = 5; FP64:
# 1 for k <= 3, 2 for k = 4, 3 for k = 5), thread u of component c
# transforms lines u, u + TPC, ... of the (2k+2)^2 lines of a pass.


def patch_threads(k, f32):
    w = ((1 if k <= 2 else (2 if k <= 4 else 3)) if f32 else (1 if k <= 3 else (2 if k == 4 else 3)))
    tpc = 32 * w
    lpc = (2 * k + 2) ** 2
    r = (lpc + tpc - 1) // tpc
    return w, tpc, r, 3 * tpc


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("f32", [True, False])
def test_patch_pass_covers_every_line_once(k, f32):
    w, tpc, r, nt = patch_threads(k, f32)
    npd = 2 * k + 2
    lpc = npd * npd
    assert nt % 32 == 0 and nt <= 1024
    for c in range(3):
        seen = np.zeros(lpc, dtype=np.int32)
        for tid in range(c * tpc, (c + 1) * tpc):
            cc, u = tid // tpc, tid - (tid // tpc) * tpc
            assert cc == c  # the component is warp-uniform: tpc is a multiple of 32
            for rr in range(r):
                line = u + rr * tpc
                if line < lpc:
                    seen[line] += 1
        assert (seen == 1).all()
    # the CTA-wide reductions use one partial per warp
    assert nt // 32 == 3 * w


# ---------------------------------------------------------------- apply kernel
# Restated from launch_apply_k and apply_velocity_kernel (apply.cu): BJ cells
# per tile side; every column cut into runs of `chunk` cells, numbered column
# by column.  FP32 and FP64 at k = 5: one run per CTA (chunk from ~8 CTAs
# per SM, runs of at least 4 cells).  FP64 up to k = 4: one wave of G CTAs
# (at least 4 cells each) marching
# whole columns; whole rounds of G runs go round-robin (CTA g takes run
# g + r G), and the cells of the remaining runs are split evenly into
# contiguous ranges in column order.

BJ = {1: 8, 2: 5, 3: 4, 4: 3, 5: 2}


def apply_grid(n, k, tuned, wave, f64, nsm=152):
    f64 = f64 and k <= 4  # the persistent march
    nd = k + 1
    m = n * nd
    tj = BJ[k] * nd
    ntile = (m + tj - 1) // tj
    tiles = ntile * ntile
    total = 3 * tiles * n
    nch = (8 * nsm + 3 * tiles - 1) // (3 * tiles)
    nch = max(1, min(nch, n // 4 if n // 4 > 0 else 1))
    chunk = min(tuned, n) if tuned > 0 else (n if f64 else (n + nch - 1) // nch)
    runs = 3 * tiles * ((n + chunk - 1) // chunk)
    grid = max(1, min(wave, total // 4)) if f64 else runs
    return m, tj, ntile, total, grid, chunk


def apply_runs(n, k, tuned, wave, f64):
    """(CTA, component, tile, cc0, cc1) of every run, as the kernel walks them."""
    m, tj, ntile, total, grid, chunk = apply_grid(n, k, tuned, wave, f64)
    f64 = f64 and k <= 4
    tiles = ntile * ntile
    ncol = 3 * tiles
    nch = (n + chunk - 1) // chunk
    rounds, f_rest = 1, ncol * n
    if f64:
        rounds = ncol * nch // grid
        u_rest = rounds * grid
        f_rest = (u_rest // nch) * n + (u_rest % nch) * chunk
    rest = ncol * n - f_rest
    runs = []
    for g in range(grid):
        for r in range(rounds):
            u = g + r * grid
            col, ch = divmod(u, nch)
            cc0 = ch * chunk
            runs.append((g, col // tiles, col % tiles, cc0, min(n, cc0 + chunk)))
        if not f64:
            continue
        f, fend = f_rest + rest * g // grid, f_rest + rest * (g + 1) // grid
        while f < fend:
            col, cc0 = divmod(f, n)
            cc1 = min(n, cc0 + (fend - f))
            f += cc1 - cc0
            runs.append((g, col // tiles, col % tiles, cc0, cc1))
    return runs


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [2, 3, 4, 6, 8, 12, 16, 24])
@pytest.mark.parametrize("tuned,wave,f64", [(0, 304, True), (0, 7, True), (0, 100000, True), (1, 304, True),
                                            (3, 304, True), (5, 7, True), (1000, 304, True), (0, 304, False),
                                            (1, 304, False), (3, 304, False), (1000, 304, False)])
def test_apply_march_writes_every_velocity_entry_once(n, k, tuned, wave, f64):
    nd = k + 1
    m, tj, ntile, total, grid, chunk = apply_grid(n, k, tuned, wave, f64)
    assert total < 2 ** 31 and grid < 2 ** 31
    # lines: the tiles cover [0, m)^2 with inactive threads past m
    lines = np.zeros((m, m), dtype=np.int32)
    for t in range(ntile * ntile):
        j0, l0 = (t % ntile) * tj, (t // ntile) * tj
        lines[j0:min(m, j0 + tj), l0:min(m, l0 + tj)] += 1
    assert (lines == 1).all()
    # along the continuous direction, per (component, tile) column: the runs'
    # written nodes plus the top node
    written = np.zeros((3, ntile * ntile, m + 1), dtype=np.int32)
    cells = 0
    for g, c, tile, cc0, cc1 in apply_runs(n, k, tuned, wave, f64):
        assert 0 <= g < grid and 0 <= c < 3 and 0 <= tile < ntile * ntile and 0 <= cc0 < cc1 <= n
        cells += cc1 - cc0
        cstart = cc0 - 1 if cc0 > 0 else 0
        for cc in range(cstart, cc1):
            if cc < cc0:
                continue  # carry-only step for the cell below the run
            written[c, tile, cc * nd: cc * nd + nd] += 1
            if cc == n - 1:
                written[c, tile, m] += 1
    assert cells == total
    assert (written == 1).all()


def test_apply_shares_are_balanced():
    # FP64, one wave of 304 resident CTAs on a 64^3, k = 3 level (768 columns
    # of 64 cells): two rounds of whole columns, then 160 columns split
    # evenly: every CTA marches 161 or 162 cells
    per, first = {}, {}
    for g, c, tile, cc0, cc1 in apply_runs(64, 3, 0, 304, True):
        per.setdefault(g, []).append((cc0, cc1))
        first.setdefault(g, []).append(c * 256 + tile)
    assert len(per) == 304
    assert {sum(b - a for a, b in v) for v in per.values()} <= {161, 162}
    assert all(v[0] == (0, 64) and v[1] == (0, 64) for v in per.values())
    # round r: CTA g marches column g + 304 r, so the CTAs of a round work on
    # neighbouring tiles
    assert all(v[:2] == [g, g + 304] for g, v in first.items())
    # FP32: 1536 CTAs of one 32-cell run each
    m, tj, ntile, total, grid, chunk = apply_grid(64, 3, 0, 304, False)
    assert (grid, chunk) == (1536, 32)


def test_apply_staging_offsets_fit_in_32_bits():
    # every mesh stk_setup accepts: n = 2^L or 3 * 2^L, n (k+1) <= 1200
    sides = sorted({s << L for s in (2, 3) for L in range(12)})
    for k in range(1, 6):
        nd = k + 1
        for n in sides:
            m = n * nd
            if m > 1200:
                continue
            for c in range(3):
                e0 = m + 1 if c == 0 else m
                e1 = m + 1 if c == 1 else m
                sc = 1 if c == 0 else (e0 if c == 1 else e0 * e1)
                d1 = 1 if c == 0 else 0
                d2 = 1 if c == 2 else 2
                s1 = 1 if d1 == 0 else e0
                s2 = e0 if d2 == 1 else e0 * e1
                # largest per-CTA offset of a staged element of cell 0
                assert nd * sc + (m - 1) * s1 + (m - 1) * s2 < 2 ** 31, (n, k, c)


# ---------------------------------------------------------------- transfers
# Restated from prolongate_add_kernel / restrict_kernel (transfer.cu): one CTA
# per coarse cell; per field the fine nodes are the lower k+1 nodes of each of
# the 8 children in every direction, the coarse nodes the cell's own nodes.


def _field(f, m):
    ext = [m + 1 if d == f else m for d in range(3)]
    nvel = (m + 1) * m * m
    return (f * nvel if f < 3 else 3 * nvel), (1, ext[0], ext[0] * ext[1]), (f if f < 3 else -1)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("nc", [1, 2, 3, 4])
def test_transfer_index_maps(nc, k):
    nd = k + 1
    mc, mf = nc * nd, 2 * nc * nd
    dc, df = Discretization(nc, k), Discretization(2 * nc, k)
    fine_writes = np.zeros(df.N, dtype=np.int32)
    coarse_adds = np.zeros(dc.N, dtype=np.int32)
    a = np.arange(nd)
    for cell in range(nc ** 3):
        pc = (cell % nc, (cell // nc) % nc, cell // (nc * nc))
        for f in range(4):
            offc, stc, cdir = _field(f, mc)
            offf, stf, _ = _field(f, mf)
            # fine nodes: every child (ch0, ch1, ch2), lower nd nodes per direction
            g = [np.add.outer(2 * pc[d] * nd + np.array([0, nd]), a).reshape(-1) for d in range(3)]
            G2, G1, G0 = np.meshgrid(g[2], g[1], g[0], indexing="ij")
            keep = np.ones(G0.shape, bool) if cdir < 0 else ((G0, G1, G2)[cdir] != 0)
            idx = offf + G0 * stf[0] + G1 * stf[1] + G2 * stf[2]
            fine_writes[idx[keep]] += 1  # each fine node appears once per CTA and field
            # coarse nodes of the cell: nd per direction, nd + 1 along the continuous one
            b = [pc[d] * nd + np.arange(nd + 1 if d == cdir else nd) for d in range(3)]
            B2, B1, B0 = np.meshgrid(b[2], b[1], b[0], indexing="ij")
            keep = np.ones(B0.shape, bool)
            if cdir >= 0:
                gcd = (B0, B1, B2)[cdir]
                keep = (gcd != 0) & (gcd != mc)
            cidx = offc + B0 * stc[0] + B1 * stc[1] + B2 * stc[2]
            assert cidx.max() < dc.N and idx.max() < df.N
            coarse_adds[cidx[keep]] += 1
    free_f, free_c = df.free_mask(), dc.free_mask()
    # prolongation: every free fine node written exactly once (plain +=, no race)
    assert (fine_writes[free_f] == 1).all() and (fine_writes[~free_f] == 0).all()
    # restriction: at most two atomic contributions onto zero (order independent)
    assert (coarse_adds[free_c] >= 1).all() and coarse_adds.max() <= 2
    assert (coarse_adds[~free_c] == 0).all()


def _planar_patch_global(j, v0, v1, k, m):
    """The 2D patch kernel's patch-local to global map (planar.cu), restated."""
    nd, npc, npd = k + 1, 2 * k + 1, 2 * k + 2
    nv, nvel = npc * npd, (m + 1) * m
    if j < nv:
        ix, iy = j % npc, j // npc
        return ((v0 - 1) * nd + 1 + ix) + (m + 1) * ((v1 - 1) * nd + iy)
    if j < 2 * nv:
        jj = j - nv
        ix, iy = jj % npd, jj // npd
        return nvel + ((v0 - 1) * nd + ix) + m * ((v1 - 1) * nd + 1 + iy)
    jj = j - 2 * nv
    ix, iy = jj % npd, jj // npd
    return 2 * nvel + ((v0 - 1) * nd + ix) + m * ((v1 - 1) * nd + iy)


@pytest.mark.parametrize("n,k", [(2, 1), (4, 3), (8, 2), (4, 8)])
def test_planar_patch_map_matches_oracle_patches(n, k):
    """The 2D patch kernel's block-to-vertex decode and patch-local map give
    the oracle's colour vertices and patch DoF sets: in bounds, no constrained
    entry, disjoint within a colour."""
    from oracle.planar import PlanarDiscretization, planar_colour_vertices, planar_patch_dofs

    d = PlanarDiscretization(n, k)
    m, nloc = n * (k + 1), 2 * (2 * k + 1) * (2 * k + 2) + (2 * k + 2) ** 2
    free = d.free_mask()
    for colour in range(4):
        cnt0 = n // 2 if colour & 1 else (n - 1) // 2
        cnt1 = n // 2 if colour & 2 else (n - 1) // 2
        verts = []
        for blk in range(cnt0 * cnt1):
            t0, t1 = blk % cnt0, blk // cnt0
            verts.append((2 * t0 + 1 if colour & 1 else 2 * t0 + 2, 2 * t1 + 1 if colour & 2 else 2 * t1 + 2))
        assert verts == planar_colour_vertices(n, colour)
        seen = set()
        for v in verts:
            g = [_planar_patch_global(j, v[0], v[1], k, m) for j in range(nloc)]
            assert sorted(g) == sorted(planar_patch_dofs(d, v).tolist())
            assert all(0 <= x < d.N and free[x] for x in g)
            assert not seen.intersection(g)
            seen.update(g)
