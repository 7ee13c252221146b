"""The scheduled sketch product A~ = A S (Algorithm 1 line 1, Lemma 3.2 item 2).

CPU part: the host plan (spm_sched_plan_host) on the oracle's sketch.  Every
entry of S must be gathered exactly once by the lane that owns its column (part),
with its sign; every step of every warp must read 32 distinct banks (or one
address several times); lanes without an entry, and idle lanes, may read only
the zero pad.  GPU part: A S through the C ABI on shapes that take the scheduled
kernel (checked with spm_sketch_plan), against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import sketch as osk

TT, LANES, PAD = 96, 1024, 32


@pytest.fixture(scope="module")
def spmlib():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    return _spm


def _columns(n, r1, s, seed):
    """Column lists of the oracle's sketch: col_ptr (r1 + 1), col_ent (j | sign bit)."""
    cols, signs = osk.sketch_entries(n, r1, s, seed)
    j = np.repeat(np.arange(n), s)
    c = cols.reshape(-1)
    neg = (signs.reshape(-1) < 0).astype(np.uint64)
    order = np.lexsort((j, c))
    ent = (j[order].astype(np.uint64) | (neg[order] << np.uint64(31))).astype(np.uint32)
    ptr = np.zeros(r1 + 1, dtype=np.int64)
    np.add.at(ptr, c + 1, 1)
    return np.cumsum(ptr), ent


def _check_plan(plan, n, r1, col_ptr, col_ent):
    G, cw = plan["groups"], plan["cw"]
    got = {}
    steps = 0
    for g in range(G):
        slots, partner = plan["slots"][g], plan["partner"][g]
        ncols = min(cw, r1 - g * cw)
        slot_col = {}
        for c in range(ncols):
            slot_col[c] = c
            if partner[c] >= 0:
                slot_col[int(partner[c])] = c
        for w in range(32):
            tp, tm = (int(x) for x in plan["wsteps"][g, w])
            assert tp >= 0 and tm >= 0 and tp + tm <= TT
            steps += tp + tm
            W = plan["words"][g, w].astype(np.int64)          # (TT/2, 32)
            for ph, T in ((0, tp), (1, tm)):
                for t in range(T):
                    r = TT - tp + t if ph == 0 else tm - 1 - t
                    off = (W[r >> 1] >> (17 if r & 1 else 0)) & 0x7FFF   # 32 lanes
                    assert not np.any(W[r >> 1] & 0x18000)            # bits 15-16 clear
                    banks = {}
                    for k in range(32):
                        o = int(off[k])
                        # one wavefront: a bank is read at one address only
                        assert banks.setdefault(o & 31, o) == o, (g, w, ph, t)
                        sl = int(slots[w * 32 + k])
                        if o < PAD:
                            continue                         # the zero pad
                        assert sl >= 0, "idle lane reads data"
                        sign = -1 if ph == 1 else 1
                        if sl & (LANES << 16):
                            sign = -sign
                        col = g * cw + slot_col[sl & 0xFFFF]
                        key = (col, o - PAD)
                        assert key not in got, "entry gathered twice"
                        got[key] = sign
    for c in range(r1):
        for e in col_ent[col_ptr[c]:col_ptr[c + 1]]:
            j, sign = int(e & 0x7FFFFFFF), (-1 if e >> 31 else 1)
            assert got.pop((c, j)) == sign
    assert not got, "gathered something that is not an entry of S"
    assert steps == plan["steps"]
    assert 32 * steps >= len(col_ent)


@pytest.mark.parametrize("n,r1,s,seed", [(4096, 500, 8, 42), (2048, 2000, 8, 5),
                                         (16384, 800, 1, 7), (1024, 40, 3, 9)])
def test_plan_covers_every_entry_once_without_bank_conflicts(spmlib, n, r1, s, seed):
    col_ptr, col_ent = _columns(n, r1, s, seed)
    plan = spmlib.sched_plan_host(n, r1, col_ptr, col_ent, search=20000)
    _check_plan(plan, n, r1, col_ptr, col_ent)


def test_plan_efficiency_on_the_bench_columns(spmlib):
    # the 16384 x 2000, s = 8 sketch: at least 80% of the wavefronts carry an entry
    n, r1, s = 16384, 2000, 8
    col_ptr, col_ent = _columns(n, r1, s, 42)
    plan = spmlib.sched_plan_host(n, r1, col_ptr, col_ent, search=300000)
    assert plan["groups"] == 2
    assert n * s / (32 * plan["steps"]) >= 0.80


def test_plan_refuses_columns_beyond_the_lane_budget(spmlib):
    # 200 entries in one column: more than two lanes' worth
    n, r1 = 256, 2
    ent = np.arange(n, dtype=np.uint32)
    col_ptr = np.array([0, 200, 256], dtype=np.int64)
    with pytest.raises(spmlib.SpmError) as e:
        spmlib.sched_plan_host(n, r1, col_ptr, ent, search=0)
    assert e.value.code == 7


# ------------------------------------------------------------------ GPU
def _dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,r1,s", [(333, 4096, 500, 8), (100, 2048, 2000, 8),
                                      (77, 16384, 800, 1), (64, 16384, 2000, 8),
                                      (40, 20000, 400, 1), (1, 1024, 40, 3),
                                      # many rows per CTA: the row ring wraps many times
                                      (3001, 4096, 1500, 8), (2000, 20000, 400, 1)])
def test_scheduled_apply_parity(spmlib, m, n, r1, s):
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n))
    So = osk.Sketch(n, r1, s, 42)
    ref = osk.apply_right(A, So)
    S = spmlib.Sketch(n, r1, s, 42)
    assert spmlib.sketch_plan(S)[0] == 0
    spmlib.sketch_set_plan(S, 1)             # plan at this (small) product
    out = spmlib.sketch_apply(S, _dev(A)).double().cpu().numpy()
    state, steps, groups = spmlib.sketch_plan(S)
    assert state == 1 and groups == -(-r1 // 1008) and 32 * steps >= n * s
    scale = np.sqrt(s) * np.abs(A).max()
    assert np.max(np.abs(out - ref)) <= 1e-5 * scale
    # a second call reuses the plan and gives the same bits
    out2 = spmlib.sketch_apply(S, _dev(A)).double().cpu().numpy()
    assert np.array_equal(out, out2)


@pytest.mark.gpu
def test_scheduled_apply_with_padded_rows(spmlib):
    # lda > n (a multiple of 4): rows start 16-byte aligned inside a wider array
    m, n, r1, s = 50, 2048, 300, 8
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, n + 12))
    S = spmlib.Sketch(n, r1, s, 11)
    spmlib.sketch_set_plan(S, 1)
    Ad = _dev(A)[:, :n]
    out = spmlib.sketch_apply(S, Ad).double().cpu().numpy()
    assert spmlib.sketch_plan(S)[0] == 1
    ref = osk.apply_right(A[:, :n], osk.Sketch(n, r1, s, 11))
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.sqrt(s) * np.abs(A).max()


@pytest.mark.gpu
def test_mixed_range_finder_reads_fro_norm_from_the_scheduled_pass(spmlib):
    # |A|_F comes from the squares the lanes gather (each element s times, over all
    # column groups, divided by s)
    m, n, r1, s = 700, 4096, 1500, 8
    rng = np.random.default_rng(4)
    A = rng.standard_normal((m, n)).astype(np.float32)
    S = spmlib.Sketch(n, r1, s, 42)
    spmlib.sketch_set_plan(S, 1)
    Q, info = spmlib.range_finder(S, _dev(A), 100, 1, omega_seed=43,
                                  precision=spmlib.PREC_MIXED)
    assert spmlib.sketch_plan(S)[0] == 1
    fro = float(np.linalg.norm(A.astype(np.float64)))
    assert abs(info["fro_a"] / fro - 1.0) < 1e-6


@pytest.mark.gpu
def test_plan_modes(spmlib):
    n, r1, s = 1024, 200, 8
    A = _dev(np.random.default_rng(9).standard_normal((64, n)))
    S = spmlib.Sketch(n, r1, s, 3)
    spmlib.sketch_apply(S, A)                # 64 x 1024 elements: below the automatic size
    assert spmlib.sketch_plan(S)[0] == 0
    spmlib.sketch_set_plan(S, 0)
    spmlib.sketch_apply(S, A)
    assert spmlib.sketch_plan(S)[0] == -1    # switched off
    spmlib.sketch_set_plan(S, 1)
    spmlib.sketch_apply(S, A)
    assert spmlib.sketch_plan(S)[0] == 1
    with pytest.raises(spmlib.SpmError):
        spmlib.sketch_set_plan(S, 0)         # the plan, once built, stays


@pytest.mark.gpu
def test_mixed_rsvd_projection_from_the_split_written_by_the_sketch_pass(spmlib):
    # In mixed precision the scheduled pass also writes A's (hi, lo) BF16 split,
    # which the projection B = Q^T A then uses instead of splitting A again.  The
    # same problem with the plan switched off (general sketch kernel, separate
    # split) must give the same approximation: sigma within 1e-4 sigma_1 and the
    # residual within 0.5% (the two sketch kernels sum in different orders).
    m, n, r1, s, k = 1500, 4096, 600, 8, 40
    rng = np.random.default_rng(12)
    Uo, _ = np.linalg.qr(rng.standard_normal((m, k + 20)))
    Vo, _ = np.linalg.qr(rng.standard_normal((n, k + 20)))
    A = (Uo * (0.9 ** np.arange(k + 20))) @ Vo.T + 1e-4 * rng.standard_normal((m, n))
    Ad = _dev(A.astype(np.float32)).float()
    res = []
    for plan in (1, 0):
        S = spmlib.Sketch(n, r1, s, 42)
        spmlib.sketch_set_plan(S, plan)
        U, sg, Vt, _ = spmlib.rsvd(S, Ad, k, 1, k, precision=spmlib.PREC_MIXED)
        assert spmlib.sketch_plan(S)[0] == (1 if plan else -1)
        U, sg, Vt = U.double().cpu().numpy(), sg.double().cpu().numpy(), Vt.double().cpu().numpy()
        res.append((sg, np.linalg.norm(A - (U * sg) @ Vt)))
    (s1, e1), (s2, e2) = res
    assert np.max(np.abs(s1 - s2)) <= 1e-4 * s2[0]
    assert abs(e1 / e2 - 1.0) <= 5e-3
