"""Host-side checks of the C ABI (no GPU): the library loads, exports every declared symbol,
and its host-only entry points (ordering, symbolic analysis, validation) agree with the oracle."""
import numpy as np
import pytest

import oracle as O
import synth
from paper_2002_05026_gb300 import _abi


@pytest.fixture(scope="module")
def lib():
    from paper_2002_05026_gb300 import build
    build.build()
    return _abi.load()


def test_exports_every_declared_symbol(lib):
    names = _abi.header_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_default_options(lib):
    o = _abi.d3m_default_options()
    assert o.precision == _abi.D3M_MIXED_BF16X3 and o.refine_tol == 1e-12 and o.max_nrhs == 32


@pytest.mark.parametrize("g", [(2, 2, 1), (3, 1, 1), (1, 3, 1), (4, 1, 1), (8, 8, 1), (6, 6, 6), (5, 3, 2), (1, 1, 1)])
def test_grid_nd_matches_oracle(lib, g):
    assert _abi.d3m_order_grid_nd(*g).tolist() == O.nd_order(*g).tolist()


def _oracle_counts(g, m, perm):
    cp, ri = synth.lower_pattern(*g)
    inv = np.empty(len(perm), dtype=int)
    inv[perm] = np.arange(len(perm))
    keys = []
    for c in range(cp.size - 1):
        for e in range(cp[c], cp[c + 1]):
            i, j = inv[ri[e]], inv[c]
            keys.append((max(i, j), min(i, j)))
    st, par = O.block_symbolic(len(perm), keys)
    return st, par


@pytest.mark.parametrize("g,m", [((2, 2, 1), 64), ((8, 8, 1), 512), ((6, 6, 6), 512), ((4, 4, 1), 100), ((3, 2, 2), 7)])
def test_analyze_matches_oracle_symbolic(lib, g, m):
    perm = O.nd_order(*g)
    cp, ri = synth.lower_pattern(*g)
    info = _abi.d3m_analyze(cp, ri, m=m, perm=perm, tile=128)
    st, par = _oracle_counts(g, m, perm)
    assert info["nblk"] == len(perm)
    assert info["nnzb_K"] == ri.size
    assert info["nblk_L_offdiag"] == sum(len(s) for s in st)
    assert info["etree_depth"] == O.etree_depth(par)
    assert info["max_col_height"] == max(len(s) for s in st)
    assert info["factor_flops"] == pytest.approx(O.factor_flops(st, m), rel=1e-12)
    assert info["n"] == len(perm) * m


def test_analyze_tile_counts_2x2(lib):
    # 2x2 grid, m = 64, tile 64: one tile per block -> tiles = blocks of L (4 diagonal + 5);
    # tile updates: col 2 gets 2 (from cols 0, 1) for (2,2), (3,2); col 3: (3,3) from 0, 1, 2
    cp, ri = synth.lower_pattern(2, 2, 1)
    info = _abi.d3m_analyze(cp, ri, m=64, perm=O.nd_order(2, 2, 1), tile=64)
    assert info["ntiles"] == 9
    # (2,0),(3,0),(2,1),(3,1): 0 updates; (2,2): 2; (3,2): 2; (3,3): 3 (k = 0, 1, 2)
    assert info["ntile_updates"] == 7


@pytest.mark.parametrize("bad", ["nodiag", "unsorted", "oob", "perm"])
def test_invalid_patterns_rejected(lib, bad):
    cp, ri = synth.lower_pattern(2, 2, 1)
    cp, ri = cp.copy(), ri.copy()
    perm = None
    if bad == "nodiag":
        ri[0] = 1
    elif bad == "unsorted":
        ri[1], ri[2] = ri[2], ri[1]
    elif bad == "oob":
        ri[-1] = 9
    else:
        perm = np.array([0, 0, 1, 2], dtype=np.int32)
    with pytest.raises(_abi.D3MError) as e:
        _abi.d3m_analyze(cp, ri, m=8, perm=perm)
    assert e.value.code == _abi.D3M_ERR_INVALID


def test_batch_create_rejects_bad_instance(lib):
    # validation happens before any device call: the error names the failing instance
    from paper_2002_05026_gb300 import D3MBatch
    cp, ri = synth.lower_pattern(2, 2, 1)
    bad = ri.copy()
    bad[-1] = 9
    with pytest.raises(_abi.D3MError) as e:
        D3MBatch([(cp, ri, 8), (cp, bad, 8)])
    assert e.value.code == _abi.D3M_ERR_INVALID
    with pytest.raises(_abi.D3MError) as e:
        D3MBatch([(cp, ri, 8), (cp[:-1], ri, 8)])
    assert e.value.code == _abi.D3M_ERR_INVALID


def test_block_diagonal_union_analysis(lib):
    # the batch is analysed as the block-diagonal union of its instances: counts add up and the
    # elimination forest is as deep as its deepest tree
    specs = [((2, 2, 1), 64), ((3, 3, 1), 32), ((4, 4, 1), 128)]
    cps, ris, perms, sizes, infos = [], [], [], [], []
    off = 0
    for g, m in specs:
        cp, ri = synth.lower_pattern(*g)
        pm = O.nd_order(*g)
        infos.append(_abi.d3m_analyze(cp, ri, m=m, perm=pm))
        cps.append(cp[1:] + (cps[-1][-1] if cps else 0))
        ris.append(ri + off)
        perms.append(pm + off)
        sizes += [m] * (cp.size - 1)
        off += cp.size - 1
    colptr = np.concatenate([[0]] + cps).astype(np.int64)
    info = _abi.d3m_analyze(colptr, np.concatenate(ris), blk_size=np.array(sizes), perm=np.concatenate(perms))
    for k in ("nblk", "nnzb_K", "nblk_L_offdiag", "ntiles", "ntile_updates", "ndep_edges"):
        assert info[k] == sum(i[k] for i in infos), k
    assert info["factor_flops"] == pytest.approx(sum(i["factor_flops"] for i in infos), rel=1e-12)
    assert info["etree_depth"] == max(i["etree_depth"] for i in infos)


def test_task_cost_model_changes_priority_set(lib):
    # the scheduler's priority lane is built from a task-duration model (Sec. II weights the dual
    # tasks with benchmarked kernel times): a measured model that makes the diagonal tasks cheaper
    # and the updates dearer moves tasks in and out of the lane; an all-zero model is the default
    from paper_2002_05026_gb300 import d3m_analyze_opts, d3m_default_options
    colptr, rowidx = synth.lower_pattern(8, 8, 1)
    perm = O.nd_order(8, 8, 1)
    base = d3m_analyze_opts(colptr, rowidx, m=512, perm=perm, opt=d3m_default_options())
    zero = d3m_default_options()
    for q in range(6):
        zero.task_cost[q] = 0.0
    assert d3m_analyze_opts(colptr, rowidx, m=512, perm=perm, opt=zero)["prio_tasks"] == base["prio_tasks"]
    meas = d3m_default_options()
    for q, v in enumerate((2500.0, 4200.0, 48000.0, 300.0, 9000.0, 4100.0)):   # ns, e.g. a fitted trace
        meas.task_cost[q] = v
    got = d3m_analyze_opts(colptr, rowidx, m=512, perm=perm, opt=meas)
    assert got["prio_tasks"] != base["prio_tasks"]
    assert got["ntiles"] == base["ntiles"] and got["factor_flops"] == base["factor_flops"]


def test_pivoting_needs_a_simt_engine(lib):
    # Bunch-Kaufman pivoting inside diagonal tiles is built in the SIMT engines only: a tensor-core
    # handle with pivot = 1 is refused at creation, before any device work
    import ctypes
    colptr, rowidx = synth.lower_pattern(2, 2, 1)
    pat, keep = _abi.make_pattern(colptr, rowidx, 16, None)
    for prec in (_abi.D3M_MIXED_BF16X3, _abi.D3M_MIXED_TF32):
        opt = _abi.d3m_default_options()
        opt.precision = prec
        opt.pivot = 1
        h = ctypes.c_void_p()
        rc = lib.d3m_create(ctypes.byref(h), ctypes.byref(pat), None, ctypes.byref(opt), None)
        assert rc == _abi.D3M_ERR_INVALID and not h
        assert b"SIMT" in lib.d3m_last_error(None)


@pytest.mark.parametrize("g,m", [((2, 2, 1), 512), ((3, 3, 1), 300), ((3, 3, 3), 200), ((8, 8, 1), 512)])
def test_tf32_paired_task_graph(lib, g, m):
    # the TF32 engine runs the source-block update segments of tiles (I, J) and (I, J + 1) as one
    # task that reads each L_IK tile once for both; the analysis builds that graph (it rejects a
    # cyclic one) with the same tiles, tile updates and flops as the unpaired graph, and the
    # shared operands remove dependency edges
    from paper_2002_05026_gb300 import d3m_analyze_opts, d3m_default_options
    colptr, rowidx = synth.lower_pattern(*g)
    perm = O.nd_order(*g)
    got = {}
    for prec in (_abi.D3M_MIXED_BF16X3, _abi.D3M_MIXED_TF32):
        opt = d3m_default_options()
        opt.precision = prec
        opt.seg_group = 8
        got[prec] = d3m_analyze_opts(colptr, rowidx, m=m, perm=perm, opt=opt)
    a, b = got[_abi.D3M_MIXED_BF16X3], got[_abi.D3M_MIXED_TF32]
    for key in ("ntiles", "ntile_updates", "factor_flops", "etree_depth"):
        assert a[key] == b[key], key
    assert b["ndep_edges"] < a["ndep_edges"]


def test_bench_engine_choice(lib):
    # bench.py --precision auto: TF32 for a throughput-bound factorization (>= 5e13 flops), the
    # split-BF16x3 engine for a smaller, critical-path-bound one; an explicit choice is kept
    import argparse
    import bench
    for wname, want in (("grid6x6x6_m512", "tf32"), ("grid8x8_m512", "bf16x3"), ("grid2x2_m64", "bf16x3")):
        w = synth.WORKLOADS[wname]
        colptr, rowidx = synth.lower_pattern(w["nx"], w["ny"], w["nz"])
        perm = O.nd_order(w["nx"], w["ny"], w["nz"])
        assert bench.resolve_precision(argparse.Namespace(precision="auto"), colptr, rowidx, w["m"], perm) == want
        assert bench.resolve_precision(argparse.Namespace(precision="simt32"), colptr, rowidx, w["m"], perm) == "simt32"


def test_task_cost_fit_counts_paired_products():
    # the autotuner's duration model from a task trace: cost = base + per * nk per task kind, where
    # a paired update task (flag 32) does 2 nk tile products
    from paper_2002_05026_gb300.autotune import fit_task_costs
    rows = []
    t = 1000
    for nk in range(1, 9):
        for flags, base, per, mult in ((4, 1500.0, 400.0, 1), (4 | 32, 1500.0, 400.0, 2), (1, 60000.0, 250.0, 1),
                                       (0, 9000.0, 120.0, 1)):
            dur = base + per * mult * nk
            rows.append([t, t + int(dur), 0, flags | (7 << 8) | (nk << 40), 0, 0, 0, 0, 0, 0])
            t += 10
    got = fit_task_costs(np.array(rows, dtype=np.int64))
    assert np.allclose(got, [1500.0, 400.0, 60000.0, 250.0, 9000.0, 120.0], rtol=1e-6, atol=1.0)


def test_recorded_traffic_follows_the_kernel_code(tmp_path):
    # bench.py reports a kernel's DRAM traffic from profiles/traffic_<workload>.txt only while the
    # record's hash matches the kernel's code: a comment edit keeps it, a code edit voids it
    import bench
    csrc = tmp_path / "paper_2002_05026_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "factor_tc.cu").write_text("// header\nint f() { return 1; }  // one\n")
    (csrc / "device.cuh").write_text("/* block\n comment */\nint g();\n")
    old_root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        sha = bench.source_sha("factor_kernel")
        (tmp_path / "profiles" / "traffic_w.txt").write_text(
            "# a comment line with several words\nfactor_kernel:tf32 123 %s\n" % sha)
        assert bench.recorded_traffic("w", "factor_kernel", "tf32") == 123.0
        assert bench.recorded_traffic("w", "factor_kernel", "bf16x3") is None
        (csrc / "factor_tc.cu").write_text("// another header\n\nint f() { return 1; }\n")
        assert bench.recorded_traffic("w", "factor_kernel", "tf32") == 123.0
        (csrc / "factor_tc.cu").write_text("int f() { return 2; }\n")
        assert bench.recorded_traffic("w", "factor_kernel", "tf32") is None
    finally:
        bench.ROOT = old_root
