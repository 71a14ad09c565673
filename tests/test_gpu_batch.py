"""Batched BSPAI-GMRES-IR (many independent systems and right-hand sides per
launch): per-system bucketing bit-exact against the oracle bucketing each
system alone, every (system, right-hand side) solution within 1e-12 of the
oracle's own solve of that system, and the full 512-system x 32-RHS batch to
forward error <= 1e-10 for every pair."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_helpers import dev, host, lib
from paper_2307_03914_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return lib()


def _system_wl(bw, s):
    A = bw["mats"][s]
    return dict(A=A, pattern=W.pattern_of(A), spai_eps=bw["spai_eps"], precs=bw["precs"], u_g="fp32", u_p="fp32",
                tau=bw["tau"], b=None, x_true=None)


def _gpu_batch(B, bw, eps=None):
    A = B.DeviceCSR.from_host(bw["A"])
    P = B.DeviceCSR.from_host(bw["pattern"], with_values=False)
    Ah = B.matrix_create(A)
    M, binfo = B.bspai_build(A, P, bw["spai_eps"])
    row_off = dev(bw["row_off"])
    BM, kinfo = B.bspai_bucket_batched(M, row_off, bw["bucket_eps"] if eps is None else eps, bw["precs"])
    Bd = dev(bw["B"].reshape(-1))
    X = torch.zeros_like(Bd)
    npairs = len(bw["mats"]) * bw["nrhs"]
    st = torch.empty(npairs, dtype=torch.int32, device="cuda")
    it = torch.empty(npairs, dtype=torch.int32, device="cuda")
    info = B.gmres_ir_solve_batched(Ah, row_off, bw["nrhs"], Bd, BM, M, X, tol=bw["tau"], pair_status=st,
                                    pair_iters=it)
    return dict(X=X, info=info, status=host(st), iters=host(it), M=M, BM=BM, kinfo=kinfo, row_off=row_off)


def test_batched_bucketing_matches_per_system_oracle(B):
    bw = W.batch_workload(nsys=7, nrhs=2, nmin=60, nmax=1500, seed=3)
    # the oracle's M of every system, stacked and handed to the library
    mufs = []
    for s in range(len(bw["mats"])):
        wl = _system_wl(bw, s)
        mufs.append(O.round_to(O.spai(wl["A"], wl["pattern"], wl["spai_eps"])["mval"], "fp32"))
    P = bw["pattern"]
    Mcsr = B.DeviceCSR(P.n, dev(P.row_ptr), dev(P.col), dev(np.concatenate(mufs)))
    M = B.M_create(Mcsr)
    row_off = dev(bw["row_off"])
    for precs, eps in [(bw["precs"], 2.0 ** -16), (["fp64", "fp32", "fp16", "e4m3", "drop"], 2.0 ** -12)]:
        BM, _ = B.bspai_bucket_batched(M, row_off, eps, precs)
        ids, stored = B.bucket_export(BM, P.nnz)
        ids, stored = host(ids), host(stored)
        off = 0
        for s, m in enumerate(bw["mats"]):
            nnz = m.nnz
            ref = O.bucket_ids(m.row_ptr, mufs[s], eps, precs)
            st, _, _ = O.bucket_store(m.row_ptr, m.col, mufs[s], ref["ids"], precs)
            assert np.array_equal(ids[off:off + nnz], ref["ids"]), (s, precs)
            assert np.array_equal(stored[off:off + nnz], st), (s, precs)
            off += nnz
        # the product on the stacked vector equals each system's own product
        x = np.random.default_rng(1).uniform(-1, 1, P.n)
        y = torch.empty(P.n, dtype=torch.float64, device="cuda")
        B.apply(BM, dev(x), y)
        yh = host(y)
        ro = bw["row_off"]
        for s, m in enumerate(bw["mats"]):
            ref = O.bucket_ids(m.row_ptr, mufs[s], eps, precs)
            st, _, _ = O.bucket_store(m.row_ptr, m.col, mufs[s], ref["ids"], precs)
            yr = O.bspmv(m.row_ptr, m.col, st, ref["ids"], precs, x[ro[s]:ro[s] + m.n])
            assert np.array_equal(yh[ro[s]:ro[s] + m.n], yr), s


def test_batched_solve_matches_oracle_per_pair(B):
    bw = W.batch_workload(nsys=6, nrhs=3, nmin=60, nmax=1200, seed=5)
    g = _gpu_batch(B, bw)
    assert g["info"]["status"] == 0 and g["info"]["converged"] == g["info"]["pairs"]
    assert np.all(g["status"] > 0)
    n = bw["A"].n
    X = host(g["X"]).reshape(bw["nrhs"], n)
    ro = bw["row_off"]
    for s, m in enumerate(bw["mats"]):
        wl = _system_wl(bw, s)
        for r in range(bw["nrhs"]):
            wl["b"] = bw["B"][r, ro[s]:ro[s] + m.n]
            xt = bw["X_true"][r, ro[s]:ro[s] + m.n]
            ref = O.solve(wl, bucket_eps=bw["bucket_eps"])
            xg = X[r, ro[s]:ro[s] + m.n]
            assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max(), (s, r)
            assert np.abs(xg - xt).max() / np.abs(xt).max() <= 1e-10
            # GMRES steps summed over the refinement steps within a few steps (the late
            # steps' counts move with the u_g summation order, see test_gpu_parity)
            assert abs(g["iters"][r * len(bw["mats"]) + s] - sum(ref["its"])) <= max(4, 0.15 * sum(ref["its"]))
        # padding rows stay zero
        assert np.all(X[:, ro[s] + m.n:ro[s + 1]] == 0)


def test_batch_of_one_equals_single_solve(B):
    bw = W.batch_workload(nsys=1, nrhs=1, nmin=900, nmax=1000, seed=7)
    g = _gpu_batch(B, bw)
    m = bw["mats"][0]
    A = B.DeviceCSR.from_host(m)
    P = B.DeviceCSR.from_host(W.pattern_of(m), with_values=False)
    M, _ = B.bspai_build(A, P, bw["spai_eps"])
    BM, _ = B.bspai_bucket(M, bw["bucket_eps"], bw["precs"])
    x = torch.empty(m.n, dtype=torch.float64, device="cuda")
    B.gmres_ir_solve(A, dev(bw["B"][0, :m.n]), BM, M, x, tol=bw["tau"])
    xb = host(g["X"])[:m.n]
    assert np.abs(xb - host(x)).max() <= 1e-12 * np.abs(host(x)).max()


def _forced(B, bw, **sched):
    B.batch_schedule_force(**sched)
    try:
        return _gpu_batch(B, bw)
    finally:
        B.batch_schedule_force(None)


@pytest.mark.parametrize("bd", [128, 512])
def test_batch_schedules_compute_the_same_bits(B, bd):
    """For a given CTA size, every MGS tile, z placement and bucket order gives the
    same solution bits, iteration counts and statuses (they move loads and storage,
    not the order of any sum); the reference schedule also matches the oracle."""
    bw = W.batch_workload(nsys=6, nrhs=3, nmin=60, nmax=1200, seed=5)
    sizes = np.diff(bw["row_off"])
    mid = int(np.sort(sizes)[len(sizes) // 2])  # z in shared memory for about half of the pairs
    ref = _forced(B, bw, block_threads=bd)
    assert ref["info"]["converged"] == ref["info"]["pairs"]
    assert ref["info"]["tuned_candidates"] == 0 and ref["info"]["block_threads"] == bd
    base = host(ref["X"])
    lo = ref["info"]["mgs_rows"]
    for sched in [dict(mgs_rows=2 * lo), dict(z_shared_rows=int(sizes.max())), dict(z_shared_rows=mid),
                  dict(m_schedule=1), dict(mgs_rows=2 * lo, z_shared_rows=mid, m_schedule=1)]:
        g = _forced(B, bw, block_threads=bd, **sched)
        for k, v in sched.items():
            assert g["info"][k] == v, (sched, g["info"])
        assert np.array_equal(host(g["X"]), base), sched
        assert np.array_equal(g["iters"], ref["iters"]) and np.array_equal(g["status"], ref["status"]), sched


@pytest.mark.parametrize("team_rows", [1024, 2048])
def test_batch_team_mode_matches_oracle_per_pair(B, team_rows):
    """Team mode: pairs on teams of ceil(n_s / team_rows) CTAs (here up to 5) with z
    in registers; every pair within 1e-12 of the oracle's own solve, GMRES counts
    within the one-CTA bars, and a second run gives the same bits."""
    bw = W.batch_workload(nsys=6, nrhs=2, nmin=300, nmax=5000, seed=21)
    g = _forced(B, bw, block_threads=512, team_rows=team_rows)
    info = g["info"]
    assert info["team_rows"] == team_rows and info["converged"] == info["pairs"], info
    sizes = np.diff(bw["row_off"])
    assert -(-sizes.max() // team_rows) >= (4 if team_rows == 1024 else 2)  # teams of several CTAs
    n = bw["A"].n
    X = host(g["X"]).reshape(bw["nrhs"], n)
    ro = bw["row_off"]
    for s, m in enumerate(bw["mats"]):
        wl = _system_wl(bw, s)
        for r in range(bw["nrhs"]):
            wl["b"] = bw["B"][r, ro[s]:ro[s] + m.n]
            xt = bw["X_true"][r, ro[s]:ro[s] + m.n]
            ref = O.solve(wl, bucket_eps=bw["bucket_eps"])
            xg = X[r, ro[s]:ro[s] + m.n]
            assert np.abs(xg - ref["x"]).max() <= 1e-12 * np.abs(ref["x"]).max(), (s, r)
            assert np.abs(xg - xt).max() / np.abs(xt).max() <= 1e-10
            assert abs(g["iters"][r * len(bw["mats"]) + s] - sum(ref["its"])) <= max(4, 0.15 * sum(ref["its"]))
        assert np.all(X[:, ro[s] + m.n:ro[s + 1]] == 0)
    g2 = _forced(B, bw, block_threads=512, team_rows=team_rows)
    assert np.array_equal(host(g2["X"]), host(g["X"])) and np.array_equal(g2["iters"], g["iters"])


def test_batch_team_mode_needs_fp32_krylov_vectors(B):
    bw = W.batch_workload(nsys=2, nrhs=1, nmin=100, nmax=200, seed=9)
    A = B.DeviceCSR.from_host(bw["A"])
    P = B.DeviceCSR.from_host(bw["pattern"], with_values=False)
    Ah = B.matrix_create(A)
    M, _ = B.bspai_build(A, P, bw["spai_eps"])
    row_off = dev(bw["row_off"])
    BM, _ = B.bspai_bucket_batched(M, row_off, bw["bucket_eps"], bw["precs"])
    Bd = dev(bw["B"].reshape(-1))
    X = torch.zeros_like(Bd)
    B.batch_schedule_force(512, team_rows=2048)
    try:
        with pytest.raises(B.BspaiError) as e:
            B.gmres_ir_solve_batched(Ah, row_off, bw["nrhs"], Bd, BM, M, X, u_g="fp64", u_p="fp64", tol=1e-8)
        assert e.value.status == B.ERR_UNSUPPORTED
    finally:
        B.batch_schedule_force(None)
    with pytest.raises(B.BspaiError):
        B.batch_schedule_force(512, team_rows=1000)


def test_batch_schedule_rejects_what_does_not_fit(B):
    bw = W.batch_workload(nsys=2, nrhs=1, nmin=100, nmax=200, seed=9)
    for sched, msg in [(dict(z_shared_rows=1 << 24), "z_shared_rows"), (dict(mgs_rows=3), "mgs_rows")]:
        with pytest.raises(B.BspaiError) as e:
            _forced(B, bw, block_threads=256, **sched)
        assert e.value.status == B.ERR_INVALID and msg in str(e.value)
    with pytest.raises(B.BspaiError):
        B.batch_schedule_force(block_threads=100)


def test_batch_autotuner_picks_the_fastest_candidate(B):
    """A new batch shape is tuned: the staged search times at least the three CTA
    sizes, the larger tile and the bucket-major order, and keeps the fastest; the
    next call of the same shape reuses it without timing."""
    bw = W.batch_workload(nsys=9, nrhs=2, nmin=200, nmax=3000, seed=13)
    g = _gpu_batch(B, bw)
    info = g["info"]
    tab = B.batch_tune_table()
    assert info["tuned_candidates"] == len(tab) >= 5, (info, tab)
    # sizes 200 .. 3000: one team size at 8,192 and 4,096 rows, so team mode is a candidate
    assert {t["team_rows"] for t in tab} >= {0, 8192, 4096}
    assert all(t["ms"] > 0 for t in tab)
    assert {t["block_threads"] for t in tab} >= {128, 256, 512}
    assert any(t["m_schedule"] == 1 for t in tab)
    best = min(tab, key=lambda t: t["ms"])
    assert (best["block_threads"], best["mgs_rows"], best["z_shared_rows"], best["m_schedule"], best["team_rows"]) == \
        (info["block_threads"], info["mgs_rows"], info["z_shared_rows"], info["m_schedule"], info["team_rows"])
    assert abs(sum(t["ms"] for t in tab) - info["tune_ms"]) <= 1e-3 * info["tune_ms"] + 1e-3
    g2 = _gpu_batch(B, bw)
    assert g2["info"]["tuned_candidates"] == 0
    assert g2["info"]["block_threads"] == info["block_threads"]
    assert np.array_equal(host(g2["X"]), host(g["X"]))


def test_batch_rejects_unaligned_offsets(B):
    bw = W.batch_workload(nsys=2, nrhs=1, nmin=100, nmax=200, seed=9)
    A = B.DeviceCSR.from_host(bw["A"])
    P = B.DeviceCSR.from_host(bw["pattern"], with_values=False)
    M, _ = B.bspai_build(A, P, 0.3)
    bad = bw["row_off"].copy()
    bad[1] -= 1
    with pytest.raises(B.BspaiError) as e:
        B.bspai_bucket_batched(M, dev(bad), 2.0 ** -16, bw["precs"])
    assert e.value.status == B.ERR_INVALID


def test_full_batch_512_systems_32_rhs(B):
    bw = W.batch_workload()
    g = _gpu_batch(B, bw)
    info = g["info"]
    assert info["pairs"] == 512 * 32 and info["converged"] == info["pairs"], info
    n = bw["A"].n
    X = g["X"].reshape(bw["nrhs"], n)
    Xt = dev(bw["X_true"])
    err = (X - Xt).abs()
    ro = bw["row_off"]
    worst = 0.0
    for s, m in enumerate(bw["mats"]):
        e = err[:, ro[s]:ro[s] + m.n].amax(dim=1)
        t = Xt[:, ro[s]:ro[s] + m.n].abs().amax(dim=1)
        worst = max(worst, float((e / t).max()))
    assert worst <= 1e-10, worst
    print("batch:", info, f"worst forward error {worst:.2e}")
