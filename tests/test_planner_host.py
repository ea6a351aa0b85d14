"""The host planner through lsmc_plan_layout_info, without a device: bump
scenarios folded onto simulated path groups, the instances (one regression
chain per scenario and strike, Sec. 2.2.1), the results (one per strike),
the job count of the backward pass for each tile shape -- the split that
gives the strikes in the money at S0 half the sub-tiles per job included --
and the device bytes a plan holds."""
import math

import pytest

from paper_2206_03719_gb300 import api, workloads
from paper_2206_03719_gb300 import build as B
from paper_2206_03719_gb300 import lsmc as L

PAPER = workloads.PAPER_FP64


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def _info(wl, sub, ppt=0):
    return api.plan_layout([wl], sub, ppt)


def _threads(precision):
    # threads per backward CTA: 64 in double, 256 in the float forms
    return 64 if precision == "fp64" else 256


def _expected_jobs(wl, subs, ppt):
    """One job per (exercise date, scenario, strike, tile); subs: the
    sub-tiles per job of each strike."""
    rounds = wl.n_steps if wl.style == "american" else 1
    tiles = sum(math.ceil(wl.n_paths / (_threads(wl.precision) * ppt * s)) for s in subs)
    return rounds * wl.n_scenarios * tiles


@pytest.mark.parametrize("greeks, groups", [
    ((), 1),
    (("delta",), 1),                      # spot bumps scale the base paths
    (("delta", "gamma"), 1),
    (("rho",), 1),                        # a rate bump is a factor exp(n dr dt) on S
    (("vega",), 3),                       # v0 +- simulates two more groups
    (("theta",), 3),                      # T +- changes the date grid
    (workloads.ALL_GREEKS, 5),            # 11 revaluations on 5 groups
])
def test_bump_scenarios_fold_onto_path_groups(lib, greeks, groups):
    wl = PAPER.replace(greeks=greeks)
    info = _info(wl, 4, 2)
    assert info.n_groups == groups
    assert info.n_instances == wl.n_scenarios * len(wl.strikes)
    assert info.n_results == len(wl.strikes)
    assert info.generated_path_steps == wl.generated_path_steps
    assert info.lsmc_path_steps == wl.lsmc_path_steps
    assert info.kernels_per_launch == 4 and info.itm_path_steps == 0 and info.d2h_bytes == 0


@pytest.mark.parametrize("precision, ppts", [("fp64", (2, 4)), ("df", (2, 4)), ("mixed", (4, 8))])
def test_backward_jobs_follow_the_tile_geometry(lib, precision, ppts):
    # a ragged path count: the last tile of every instance is partial
    wl = PAPER.replace(precision=precision, n_paths=100_003, n_steps=50)
    for ppt in ppts:
        for sub in (1, 3, 16, 64):
            info = _info(wl, sub, ppt)
            assert info.backward_jobs == _expected_jobs(wl, [sub] * len(wl.strikes), ppt)
    # a European request regresses nothing: one round of jobs (the estimator)
    eu = wl.replace(style="european")
    assert _info(eu, 8, ppts[0]).backward_jobs == _expected_jobs(eu, [8] * 5, ppts[0])


def test_in_the_money_strikes_take_half_the_sub_tiles(lib):
    # puts struck above S0 = 100 (110, 120): jobs of 16 sub-tiles, the others 32
    half = L.LSMC_SUB_ITM_HALF
    info = _info(PAPER, 32 | half, 2)
    assert info.backward_jobs == _expected_jobs(PAPER, [32, 32, 32, 16, 16], 2)
    # 131,072 paths fill whole tiles: exactly 7/5 of the uniform count
    assert 5 * info.backward_jobs == 7 * _info(PAPER, 32, 2).backward_jobs
    # calls: the strikes below S0 (80, 90)
    call = PAPER.replace(option="call")
    assert _info(call, 32 | half, 2).backward_jobs == _expected_jobs(call, [16, 16, 32, 32, 32], 2)
    # at least one sub-tile per job
    assert _info(PAPER, 1 | half, 2).backward_jobs == _info(PAPER, 1, 2).backward_jobs
    # a single strike, or strikes all out of the money: no split
    for wl in (PAPER.replace(strikes=[120.0]), PAPER.replace(strikes=[80.0, 90.0])):
        assert _info(wl, 8 | half, 2).backward_jobs == _info(wl, 8, 2).backward_jobs
    # smaller jobs keep more tile partials, all else equal
    assert info.device_bytes > _info(PAPER, 32, 2).device_bytes


def test_a_book_plan_is_the_sum_of_its_contracts(lib):
    # 128 uneven contracts of the 512-contract book in one plan: results,
    # instances, path-steps and jobs add up over the contracts (each with
    # its own date count: a regression chain per scenario of every contract)
    book = workloads.book(n_contracts=128, precision="df")
    reqs = [api.Request(w).c for w in book]
    info = L.lsmc_plan_layout_info(None, reqs, 4, 2)
    assert info.n_results == len(book)
    assert info.n_instances == sum(w.n_scenarios for w in book)
    assert info.n_groups == 5 * len(book)
    assert info.lsmc_path_steps == sum(w.lsmc_path_steps for w in book)
    assert info.backward_jobs == sum(_expected_jobs(w, [4], 2) for w in book)
    # single-strike contracts: the in-the-money split changes nothing
    assert L.lsmc_plan_layout_info(None, reqs, 4 | L.LSMC_SUB_ITM_HALF, 2).backward_jobs == \
        info.backward_jobs
    # one plan holds one precision
    mixed = reqs[:2] + [api.Request(book[2].replace(precision="fp64")).c]
    with pytest.raises(L.LsmcError) as e:
        L.lsmc_plan_layout_info(None, mixed, 4, 2)
    assert e.value.status == L.LSMC_ENOTIMPL


def test_layout_bytes_match_the_footprint(lib):
    for wl in (PAPER, PAPER.replace(precision="mixed"), workloads.SMALL_FP64):
        fp = L.lsmc_request_footprint(None, api.Request(wl).c)
        info = _info(wl, 1, 0)
        assert fp == (info.device_bytes + 255) // 256 * 256
        # larger jobs: fewer tile partials, never more bytes
        assert _info(wl, 8, 0).device_bytes <= info.device_bytes
    # the tables uploaded per plan: the end-to-end copy of the paper book
    assert _info(PAPER, 8, 4).h2d_bytes == 18688


def test_layout_query_rejects_bad_shapes(lib):
    req = [api.Request(PAPER).c]
    for sub, ppt in ((0, 0), (L.LSMC_SUB_ITM_HALF, 2), (65, 2), (8 | 0x4000, 2), (8, 3)):
        with pytest.raises(L.LsmcError) as e:
            L.lsmc_plan_layout_info(None, req, sub, ppt)
        assert e.value.status == L.LSMC_EINVAL
    with pytest.raises(L.LsmcError) as e:
        L.lsmc_plan_layout_info(None, [api.Request(PAPER.replace(n_paths=0)).c], 8, 2)
    assert e.value.status == L.LSMC_EINVAL
