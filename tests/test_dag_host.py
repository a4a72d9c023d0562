"""Host tables of the dependency-driven sweeps, no GPU needed.

Section 4.3.3 puts a barrier between consecutive colors of a substitution.
The dependency-driven sweeps (sweep_kernel 8) let a level-1 block wait only
for the level-1 blocks its other-color couplings read (Eq. "for3"), or for
a whole color's completion counter where it reads more than 16 of that
color's level-1 blocks, and they add a row's terms in rounds as the list is
published.  A wait list that missed a source would be a race the bitwise GPU
tests could pass by chance, so the lists hbmc_build makes (hbmc_get_dag_deps,
host_only contexts) are checked here against the reordered matrix itself:

  - complete: every level-1 block a level-1 block reads is listed, or its
    color's counter is;
  - only sources: every listed level-1 block is read, a color is listed
    exactly when more than 16 of its level-1 blocks are read, and nothing of
    the level-1 block's own color or of a later color in the sweep is listed;
  - in gathering order, so that after any prefix of the list is published,
    every term the kernel then treats as readable (forward: column below the
    first row of the next unpublished entry; backward: column at or above
    the row after its last) has its source in that prefix.
"""
import numpy as np
import pytest

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

COLOR_WAIT = 16  # more level-1 blocks of one color read than this: wait on its counter

CASES = [
    ("poisson7_8_bs8", lambda: W.poisson7(8), 8, (2, 2, 2)),
    ("poisson7_9_bs4", lambda: W.poisson7(9), 4, (1, 2, 2)),
    ("hetero27_12_rand", lambda: W.permute_input(W.heterogeneous_stencil(12, 27, 2.0, 1),
                                                 W.random_order(2, 1728)), 8, None),
    ("veclap_7_rand", lambda: W.permute_input(W.vector_laplacian(7, 3), W.random_order(4, 1029)), 8, None),
    ("hetero27_10_rand_bs32", lambda: W.permute_input(W.heterogeneous_stencil(10, 27, 1.0, 5),
                                                      W.random_order(6, 1000)), 32, None),
    # one unknown per block: many colors, and each level-1 block reads level-1
    # blocks of most earlier colors
    ("hetero27_16_rand_bs1", lambda: W.permute_input(W.heterogeneous_stencil(16, 27, 2.0, 1),
                                                     W.random_order(2, 4096)), 1, None),
    # about 37 level-1 blocks per color at bs 8: counters and single flags mixed
    ("hetero27_60_rand", lambda: W.permute_input(W.heterogeneous_stencil(60, 27, 2.0, 1),
                                                 W.random_order(2, 216000)), 8, None),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def _terms(rp, ci, R, fwd):
    """(row, column, reading level-1 block, source level-1 block) of every
    other-color coupling a sweep gathers: below the diagonal for the forward
    sweep, above it for the backward one, outside the row's own level-1 block."""
    rows = np.repeat(np.arange(len(rp) - 1, dtype=np.int64), np.diff(rp))
    cols = ci.astype(np.int64)
    keep = (cols < rows) if fwd else (cols > rows)
    rows, cols = rows[keep], cols[keep]
    u, v = rows // R, cols // R
    other = u != v
    return rows[other], cols[other], u[other], v[other]


def _check_direction(ptr, dep, rp, ci, R, tile_color, tile_ptr, fwd):
    ntiles = len(tile_color)
    nc = len(tile_ptr) - 1
    assert ptr.shape == (ntiles + 1,) and ptr[0] == 0 and ptr[-1] == len(dep)
    assert np.all(np.diff(ptr) >= 0)
    _, cols, u_of, v_of = _terms(rp, ci, R, fwd)
    order = np.lexsort((cols, u_of))
    cols, u_of, v_of = cols[order], u_of[order], v_of[order]
    starts = np.searchsorted(u_of, np.arange(ntiles + 1))
    counter_waits = 0
    for u in range(ntiles):
        ent = dep[ptr[u]:ptr[u + 1]].astype(np.int64)
        assert len(np.unique(ent)) == len(ent), f"level-1 block {u}: duplicate entries"
        tc = cols[starts[u]:starts[u + 1]]
        tv = v_of[starts[u]:starts[u + 1]]
        read = np.unique(tv)
        read_colors, per_color = np.unique(tile_color[read], return_counts=True)
        blocks = ent[ent >= 0]
        colors = -ent[ent < 0] - 1
        counter_waits += len(colors)
        # sources only, of earlier colors in this sweep's order
        assert np.all(np.isin(blocks, read)), f"level-1 block {u} waits on a level-1 block it does not read"
        assert np.all(colors < nc) and np.all(colors >= 0)
        cu = tile_color[u]
        ecol = np.concatenate([tile_color[blocks], colors])
        assert np.all(ecol < cu) if fwd else np.all(ecol > cu), f"level-1 block {u}: wait outside the sweep's order"
        # a color's counter exactly when more than COLOR_WAIT of its level-1 blocks are read
        assert set(colors.tolist()) == set(read_colors[per_color > COLOR_WAIT].tolist()), u
        assert not np.any(np.isin(tile_color[blocks], colors)), u
        # complete: each source listed itself or through its color
        covered = np.isin(read, blocks) | np.isin(tile_color[read], colors)
        assert np.all(covered), f"level-1 block {u} reads {read[~covered]} without waiting for them"
        # gathering order: strictly increasing first row (forward) / decreasing end row (backward)
        first = np.where(ent >= 0, ent, tile_ptr[np.clip(-ent - 1, 0, nc - 1)]) * R
        end = np.where(ent >= 0, ent + 1, tile_ptr[np.clip(-ent - 1, 0, nc - 1) + 1]) * R
        key = first if fwd else -end
        assert np.all(np.diff(key) > 0), f"level-1 block {u}: entries out of gathering order"
        # after publishing entries [0, k), the terms below / above the bound of entry k are covered
        src_entry = np.full(len(tv), -1, dtype=np.int64)
        pos_block = {int(b): i for i, b in enumerate(ent) if b >= 0}
        pos_color = {int(-b - 1): i for i, b in enumerate(ent) if b < 0}
        for i, v in enumerate(tv):
            src_entry[i] = pos_block.get(int(v), pos_color.get(int(tile_color[v]), -1))
        assert np.all(src_entry >= 0)
        for k in range(len(ent) + 1):
            if fwd:
                readable = tc < (first[k] if k < len(ent) else np.iinfo(np.int64).max)
            else:
                readable = tc >= (end[k] if k < len(ent) else -1)
            assert np.all(src_entry[readable] < k), \
                f"level-1 block {u}: a term treated as readable after {k} entries has an unpublished source"
    return counter_waits


@pytest.mark.parametrize("name,mk,bs,box", CASES)
def test_dag_wait_lists(lib, name, mk, bs, box):
    A = mk()
    ctx = H.hbmc_build(A, bs, 32, box=box, host_only=True)
    try:
        inf = ctx.info()
        R = bs * 32
        rp, ci, _ = H.hbmc_get_matrix(ctx)
        _, color_ptr, _, _ = H.hbmc_get_ordering(ctx)
        assert color_ptr[-1] == inf["n_pad"] and np.all(color_ptr % R == 0)
        tile_ptr = color_ptr // R
        ntiles = int(tile_ptr[-1])
        assert ntiles == inf["ntiles"]
        tile_color = np.repeat(np.arange(inf["nc"]), np.diff(tile_ptr))
        waits = 0
        for direction, fwd in ((0, True), (1, False)):
            ptr, dep = H.hbmc_get_dag_deps(ctx, direction)
            waits += _check_direction(ptr, dep, rp, ci, R, tile_color, tile_ptr, fwd)
        if name == "hetero27_60_rand":
            assert waits > 0, "the case was chosen to exercise color counters"
        if inf["nc"] == 2:
            # two colors: the first color's level-1 blocks wait for nothing going forward
            ptr, _ = H.hbmc_get_dag_deps(ctx, 0)
            assert np.all(np.diff(ptr)[: int(tile_ptr[1])] == 0)
    finally:
        ctx.close()


def test_dag_deps_arguments(lib):
    A = W.poisson7(6)
    ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2), host_only=True)
    try:
        for bad in (-1, 2):
            with pytest.raises(H.HbmcError, match="dir must be 0"):
                H.hbmc_get_dag_deps(ctx, bad)
        import ctypes
        count = ctypes.c_int64(-1)
        assert lib.hbmc_get_dag_deps(ctx.handle, 1, None, None, 0, ctypes.byref(count)) == H.OK
        assert count.value > 0
        dep = np.empty(count.value, dtype=np.int32)
        # a cap below the entry count is refused, and the count is still reported
        assert lib.hbmc_get_dag_deps(ctx.handle, 1, None, dep.ctypes.data, count.value - 1,
                                     ctypes.byref(count)) == H.ERR_INVALID_ARG
        assert count.value == len(dep)
    finally:
        ctx.close()
    ctx = H.hbmc_build(A, 8, 16, box=(2, 2, 2), host_only=True)
    try:
        with pytest.raises(H.HbmcError, match="need w = 32"):
            H.hbmc_get_dag_deps(ctx, 0)
    finally:
        ctx.close()


def test_checker_catches_planted_mistakes(lib):
    """The checks above fail on lists with a planted mistake: a dropped
    source, two entries swapped, a wait on the level-1 block's own color."""
    A = W.permute_input(W.heterogeneous_stencil(12, 27, 2.0, 1), W.random_order(2, 1728))
    ctx = H.hbmc_build(A, 8, 32, host_only=True)
    try:
        inf = ctx.info()
        R = 8 * 32
        rp, ci, _ = H.hbmc_get_matrix(ctx)
        _, color_ptr, _, _ = H.hbmc_get_ordering(ctx)
        tile_ptr = color_ptr // R
        tile_color = np.repeat(np.arange(inf["nc"]), np.diff(tile_ptr))
        ptr, dep = H.hbmc_get_dag_deps(ctx, 0)
        _check_direction(ptr, dep, rp, ci, R, tile_color, tile_ptr, True)
        u = int(np.argmax(np.diff(ptr)))  # the level-1 block with the longest list
        assert ptr[u + 1] - ptr[u] >= 2

        dropped = np.delete(dep, ptr[u])
        ptr_d = ptr.copy()
        ptr_d[u + 1:] -= 1
        swapped = dep.copy()
        swapped[ptr[u]], swapped[ptr[u] + 1] = dep[ptr[u] + 1], dep[ptr[u]]
        own = dep.copy()
        own[ptr[u]] = -(int(tile_color[u]) + 1)
        for p, d in ((ptr_d, dropped), (ptr, swapped), (ptr, own)):
            with pytest.raises(AssertionError):
                _check_direction(p, d, rp, ci, R, tile_color, tile_ptr, True)
    finally:
        ctx.close()


def _random_spd(n, density, seed, hubs):
    """A random symmetric pattern with a few dense rows and a strictly
    dominant diagonal (CSR, sorted columns)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=seed).tolil()
    for h in rng.choice(n, size=min(n, hubs), replace=False):
        M[h, rng.choice(n, size=max(1, n // 3), replace=False)] = 1.0
    S = (M + M.T).tocsr()
    S.setdiag(0.0)
    S.eliminate_zeros()
    S.data = -np.abs(S.data) - 0.1
    S = (S + sp.identity(n) * (abs(S).sum(axis=1).max() + 1.0)).tocsr()
    S.sort_indices()
    return W.CSR(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


def test_dag_wait_lists_random_patterns(lib):
    """The same checks over random sparse patterns with dense rows, random
    block sizes and algebraic blocking."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    @settings(max_examples=30, deadline=None)
    @given(st.integers(1, 900), st.floats(0.0, 0.03), st.integers(0, 2**31 - 1), st.integers(0, 4),
           st.sampled_from([1, 2, 3, 4, 8]))
    def check(n, density, seed, hubs, bs):
        A = _random_spd(n, density, seed, hubs)
        ctx = H.hbmc_build(A, bs, 32, host_only=True)
        try:
            inf = ctx.info()
            R = bs * 32
            rp, ci, _ = H.hbmc_get_matrix(ctx)
            _, color_ptr, _, _ = H.hbmc_get_ordering(ctx)
            tile_ptr = color_ptr // R
            tile_color = np.repeat(np.arange(inf["nc"]), np.diff(tile_ptr))
            for direction, fwd in ((0, True), (1, False)):
                ptr, dep = H.hbmc_get_dag_deps(ctx, direction)
                _check_direction(ptr, dep, rp, ci, R, tile_color, tile_ptr, fwd)
        finally:
            ctx.close()

    check()
