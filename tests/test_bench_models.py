"""The roofline work models of bench.py on CPU: the odd-even SAP flop count
against a term-by-term recount for 4^4 blocks, the interior-hop average for
other block shapes, and the vector bytes of the pair-arithmetic Arnoldi steps
against an explicit sum over the steps of the cycles."""
import bench


def test_odd_even_sap_flops_per_site_4x4x4x4():
    # 4^4 blocks: 6 of 8 hops per site stay inside the block on average
    H = 6.0
    hop, diag, dinv, mr = 168, 600, 576, 192
    residual = 8 * hop + diag + 24
    rhs = (dinv + H * hop + 24) / 2
    step = (2 * H * hop + dinv + diag + mr) / 2
    final = (H * hop + dinv) / 2 + 24
    expect = residual + rhs + 4 * step + final
    assert bench.sap_oe_flops_per_site((4, 4, 4, 4), 4) == expect == 10356.0
    # more MR steps cost exactly one step each
    assert bench.sap_oe_flops_per_site((4, 4, 4, 4), 5) - expect == step


def test_interior_hops_of_other_block_shapes():
    # 2 x 4 x 4 x 4: in T only one of the two hops of a site stays inside
    f2 = bench.sap_oe_flops_per_site((2, 4, 4, 4), 0)
    f4 = bench.sap_oe_flops_per_site((4, 4, 4, 4), 0)
    # H drops from 6 to 5.5: (168 + 168 / 2) per 0.5 hop in the terms with H
    assert abs((f4 - f2) - 0.5 * (168 / 2 + 168 / 2)) < 1e-9


def test_pair_arnoldi_bytes_per_cycle():
    wl = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    V = 1
    for n in wl["L"]:
        V *= n
    outer = {"iters": 11, "restart": 4, "rhs": 6, "steps": 1}
    m = bench.roofline_model("blas_fine", wl, units=6 * 98, launches=98, outer=outer, peaks={"hbm_gbs": 6795.1})
    assert m["bound"] == "hbm"
    per_rhs = 0
    for kc in (4, 4, 3):  # 11 iterations in cycles of at most 4
        per_rhs += sum(16 * (3 * k + 7) for k in range(1, kc + 1)) + 8 * kc + 32
    assert abs(m["work"] * 98 - per_rhs * 12 * V * 6) < 1e-3 * m["work"]
