"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
function include/planc.h declares, and its host-only planning calls agree
with the paper (Fig. DT) and with the oracle's statement of the split rule.
"""

import os
import re

import numpy as np
import pytest

import oracle as o

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _planc():
    lib = os.path.join(ROOT, "paper_1909_01149_gb300", "lib", "libplanc.so")
    if not os.path.exists(lib):
        from paper_1909_01149_gb300 import build
        build.build()
    from paper_1909_01149_gb300 import planc
    return planc


def test_library_exports_every_declared_function():
    planc = _planc()
    names = planc.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(planc.lib, name), f"libplanc.so does not export {name}"


def test_header_declarations_are_extern_c_plain_types():
    txt = open(os.path.join(ROOT, "include", "planc.h")).read()
    assert 'extern "C"' in txt
    for banned in ("torch", "at::Tensor", "std::"):
        assert banned not in txt


@pytest.mark.parametrize("dims", [(512, 512, 512), (64, 64, 64), (128, 128, 200, 100),
                                  (96, 96, 96, 96), (10, 1000), (1000, 10), (2, 3, 4, 5, 6),
                                  (1, 1, 7), (7, 1, 1), (384, 384, 384, 384), (3, 1000, 2, 2)])
def test_plan_split_matches_oracle_rule(dims):
    planc = _planc()
    assert planc.plan_split(dims) == o.choose_split(dims)


def test_plan_split_rejects_bad_shapes():
    planc = _planc()
    with pytest.raises(planc.PlancError):
        planc.plan_split((5,))
    with pytest.raises(planc.PlancError):
        planc.plan_split((5, 0, 3))


def _edges(text):
    return sorted(l.strip() for l in text.splitlines()
                  if l.startswith("PM") or l.startswith("mTTV"))


def test_dimension_tree_matches_fig_dt():
    planc = _planc()
    gold = open(os.path.join(HERE, "golden", "fig_dt_n5.txt")).read()
    N = int(re.search(r"^N (\d+)", gold, re.M).group(1))
    S = int(re.search(r"^S (\d+)", gold, re.M).group(1))
    got = planc.describe(tuple([8] * N), S)
    assert _edges(got) == _edges(gold)


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_dimension_tree_has_two_pms_and_every_leaf(N):
    """Two partial MTTKRPs per outer iteration for any N (Sec. 6.2) and one
    leaf per mode."""
    planc = _planc()
    for S in range(1, N):
        text = planc.describe(tuple([4] * N), S)
        e = _edges(text)
        assert sum(1 for l in e if l.startswith("PM")) == 2
        leaves = set()
        for line in e:
            dst = line.split("->")[1].strip()
            if "," not in dst:
                leaves.add(int(dst.strip("{}")))
        # a branch with one mode is its own leaf (the PM output itself)
        if S == 1:
            leaves.add(1)
        if N - S == 1:
            leaves.add(N)
        assert leaves == set(range(1, N + 1))


def test_option_defaults_cross_the_abi():
    """The binding's ctypes mirrors of the option structs agree with the C
    layout: the library's defaults read back field by field."""
    planc = _planc()
    n = planc.lib.planc_nls_opts_default()
    assert (n.mu_eps, n.admm_max_inner, n.admm_tol, n.bpp_max_iter, n.pgd_steps,
            n.nes_max_inner, n.nes_tol) == (1e-16, 5, 1e-2, 0, 1, 20, 1e-3)
    s = planc.lib.planc_solve_opts_default()
    assert (s.alg, s.iters, s.tol, s.use_graph, s.profile, s.nes_accel) == (1, 10, 0.0, 1, 0, 1)
    assert s.batch_persistent == 1  # the batched solve as one persistent launch by default
    assert s.nls.nes_max_inner == 20 and s.nls.nes_tol == 1e-3
    assert planc.ALGS["nes"] == 6 and planc.ALGS["ucp"] == 5


def test_dimension_tree_of_nmf_is_two_leaves():
    """N = 2 (NMF): the root split is S = 1 and both partial MTTKRPs are the
    leaves themselves (M^(1) = X H^(2), M^(2) = X^T H^(1)); no multi-TTV."""
    planc = _planc()
    for dims in [(300, 200), (7, 1000), (1000, 7)]:
        text = planc.describe(dims)
        assert "split S=1" in text
        assert sorted(_edges(text)) == ["PM {1,2} -> {1}", "PM {1,2} -> {2}"]


def _paper_facts():
    kv = {}
    for line in open(os.path.join(HERE, "golden", "paper_facts.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            kv[k] = int(v)
    return kv


def test_defaults_follow_the_numbers_the_paper_states():
    """ADMM at most 5 inner steps (Sec. 4.3.4), NES at most 20 (Sec. 4.3.5),
    two partial MTTKRPs per outer iteration for any N (Sec. 4.2): in the
    library's defaults, in the oracle, and in the planned dimension tree."""
    import inspect
    planc = _planc()
    facts = _paper_facts()
    d = planc.lib.planc_nls_opts_default()
    assert d.admm_max_inner == facts["admm_max_inner"]
    assert d.nes_max_inner == facts["nes_max_inner"]
    assert o.NES_MAX_INNER == facts["nes_max_inner"]
    assert inspect.signature(o.nls_admm).parameters["max_inner"].default == facts["admm_max_inner"]
    for dims in [(8, 9), (5, 6, 7), (3, 4, 5, 6), (2, 3, 4, 5, 6)]:
        pms = [e for e in _edges(planc.describe(dims)) if e.startswith("PM")]
        assert len(pms) == facts["pm_per_outer_iteration"], dims


def test_binding_rejects_bad_buffers_before_the_library():
    """The binding checks every buffer it passes as a raw pointer (device,
    dtype, contiguity, size) and raises ValueError before any library call,
    so a wrong tensor never reaches a kernel.  Runs on the host: a Context
    shell with no library handle, CPU tensors standing for device ones."""
    import torch
    planc = _planc()
    ctx = object.__new__(planc.Context)
    ctx.h = None
    ctx.dims, ctx.N, ctx.R = (6, 7, 8), 3, 4
    ctx.fdtype, ctx.device = torch.float32, torch.device("cpu")
    H = [torch.zeros(d, 4) for d in ctx.dims]
    cases = [
        lambda: ctx.mttkrp(H, 0),                                    # host factors
        lambda: ctx.gram(torch.zeros(6, 4)),
        lambda: ctx.gram(torch.zeros(24)),                           # not 2-D
        lambda: ctx.normalize(torch.zeros(6, 4)),
        lambda: ctx.nls_update("hals", torch.zeros(4, 4, dtype=torch.float64),
                               torch.zeros(6, 4), torch.zeros(6, 4)),
        lambda: ctx.gram_hadamard(torch.zeros(3, 4, 4, dtype=torch.float64), 0),
        lambda: ctx.fit(H, torch.ones(4, dtype=torch.float64)),
        lambda: ctx.partial_mttkrp(H, 0, torch.zeros(4)),
        lambda: ctx.cp_grad(H),
    ]
    for call in cases:
        with pytest.raises(ValueError):
            call()
    # the buffer check itself: each property rejects on its own
    ok = torch.zeros(16, dtype=torch.float64)
    for bad, why in [([0.0] * 16, "torch tensor"),
                     (torch.zeros(16), "dtype"),
                     (torch.zeros(15, dtype=torch.float64), "at least 16"),
                     (torch.zeros(4, 4, dtype=torch.float64).t(), "contiguous"),
                     (ok, "CUDA")]:
        with pytest.raises(ValueError, match=why):
            planc._check_buf(bad, 16, torch.float64, "x")


def test_every_computational_entry_point_cites_the_paper():
    """Each call that computes a step of the method cites the section,
    algorithm or equation it implements in its header comment; the helpers
    (status, defaults, getters) and the library's own extensions are the only
    uncited declarations, and the extensions say they have no counterpart."""
    txt = open(os.path.join(ROOT, "include", "planc.h")).read()
    decl = re.compile(r"/\*((?:(?!\*/).)*)\*/\s*(?:const\s+)?[\w\*]+\s+\**(planc_\w+)\s*\(", re.S)
    cited, uncited = set(), {}
    for comment, name in decl.findall(txt):
        if re.search(r"\b(Sec|Alg|Eq|Fig|Tab)\.", comment):
            cited.add(name)
        else:
            uncited[name] = comment
    helpers = {"planc_status_str", "planc_last_error", "planc_nls_opts_default",
               "planc_solve_opts_default", "planc_destroy", "planc_get_split",
               "planc_pm_tensor_cores", "planc_batch_schedule", "planc_batch_plan"}
    extensions = {"planc_sqnorm_noalloc"}
    assert set(uncited) <= helpers | extensions, sorted(set(uncited) - helpers - extensions)
    for name in extensions:
        assert "no counterpart" in " ".join(re.sub(r"\n\s*\*", " ", uncited[name]).split())
    for name in ("planc_init", "planc_mttkrp", "planc_mttkrp_all", "planc_partial_mttkrp",
                 "planc_gram_hadamard", "planc_gram", "planc_nls_update", "planc_normalize",
                 "planc_fit", "planc_nncp_solve", "planc_sqnorm", "planc_cp_grad",
                 "planc_batch_solve", "planc_plan_split", "planc_describe"):
        assert name in cited, name
    assert cited | set(uncited) == set(_planc().header_functions())


def test_batch_plan_deals_every_instance_longest_first():
    """The persistent batched launch's deal (host-only): every instance in
    exactly one cluster; each cluster's list in non-increasing estimated cost
    (the order it solves them); the estimate is elements x 2 x the padded
    rank class + 8e6; the greedy rule (longest first onto the least-loaded
    cluster) keeps every cluster within one instance's cost of the least
    loaded; the same input gives the same deal."""
    planc = _planc()
    rng = np.random.default_rng(5)
    shapes = [(tuple(int(v) for v in rng.integers(32, 161, 3)), int(rng.integers(8, 33)))
              for _ in range(256)]

    def cost(dims, R):
        rc = 8 if R <= 8 else 16 if R <= 16 else 32
        return dims[0] * dims[1] * dims[2] * 2.0 * rc + 8e6

    for ncl in (1, 7, 38, 256):
        lists, loads = planc.batch_plan(shapes, ncl)
        assert len(lists) == ncl
        assert sorted(b for l in lists for b in l) == list(range(len(shapes)))
        costs = [cost(*s) for s in shapes]
        for l, ld in zip(lists, loads):
            assert all(costs[a] >= costs[b] for a, b in zip(l, l[1:]))
            assert ld == pytest.approx(sum(costs[b] for b in l), rel=1e-12)
        assert max(loads) - min(loads) <= max(costs) + 1e-6 * max(loads)
        assert planc.batch_plan(shapes, ncl) == (lists, loads)
    # the benchmark batch's deal is within 3 % of perfect balance
    _, loads = planc.batch_plan(shapes, 38)
    assert max(loads) <= 1.03 * (sum(loads) / len(loads))


def test_batch_plan_rejects_bad_arguments():
    planc = _planc()
    with pytest.raises(planc.PlancError):
        planc.batch_plan([((4, 5, 6), 3)], 2)      # more clusters than instances
    with pytest.raises(planc.PlancError):
        planc.batch_plan([((4, 0, 6), 3)], 1)      # an empty mode
    with pytest.raises(planc.PlancError):
        planc.batch_plan([((4, 5, 6), 0)], 1)      # rank 0
