"""Host-side logic of bench.py (no GPU): flop and byte models, the digit budget of
the tensor-core Schur product, the default workload and the argument parser."""
import numpy as np

import bench


def test_flop_split_keeps_the_total():
    for d, p in ((2, 1), (2, 2), (3, 2), (3, 3)):
        a = bench.flop_counts(d, p, sum_factorised=True)
        b = bench.flop_counts(d, p, sum_factorised=True, tc_schur=True)
        assert a["total"] == b["total"] and b["elim"] + b["schur"] == a["elim"]
        m, n1 = d + 2, p + 1
        NU, NT = m * n1 ** d, 2 * d * m * n1 ** (d - 1)
        assert b["schur"] == 2 * NT * NT * NU


def test_ozaki_digit_budget():
    """5 K (2^b - 1)^2 < 2^24 (the groups k <= 6 accumulate exactly in FP32), b s >= 54,
    and b the largest such width; hex p = 2 and p = 3 take (7, 8) and (6, 9)."""
    for K in (16, 36, 40, 64, 135, 320):
        b, s = bench.ozaki_digits(K)
        assert 5 * K * (2 ** b - 1) ** 2 < 2 ** 24 and b * s >= 54 and b * (s - 1) < 54
        assert b == 8 or 5 * K * (2 ** (b + 1) - 1) ** 2 >= 2 ** 24
    assert bench.ozaki_digits(135) == (7, 8) and bench.ozaki_digits(320) == (6, 9)


def test_recover_bytes_models():
    hex_b = bench.hex_recover_bytes(3, 2, 4096)
    NU, NT, NQV = 135, 270, 405
    assert hex_b == 8.0 * 4096 * (NU * (NT + 1) + NU * (NU + 1) / 2 + NQV + NT + NU + NQV)
    layout = {"face_p": np.array([1, 2, 3, 4]), "e2f": np.array([[0, 1, 2, 3]])}
    tb = bench.tet_recover_bytes(layout, np.array([4]))
    Np, sfp = 35, 3 + 6 + 10 + 15
    NU, t = 5 * Np, 5 * sfp
    assert tb == 8.0 * (NU * (t + 1) + NU * (NU + 1) / 2 + 3 * Np * Np + 3 * Np * sfp + 3 * NU + t + 4 * NU)


def test_default_workload_is_the_tetrahedral_mesh():
    assert bench.DEFAULT_WORKLOAD == "tet-p1to4-30x20x28-curved"
    assert bench.WORKLOADS[bench.DEFAULT_WORKLOAD]["kind"] == "tet"
    assert bench.TET_DRAM_BYTES_PER_ELEMENT > 1e6
    peak, src = bench.hbm_peak_gbs()
    assert peak > 1000 and isinstance(src, str)


def test_oracle_check_elements_cover_every_degree():
    """The bench's oracle check takes the first and last element of every degree of a
    mixed-degree mesh, and four spread elements (ends included) of a uniform one."""
    elem_p = np.array([2, 1, 1, 4, 2, 3, 4, 1])
    ids = bench.oracle_check_elements(elem_p=elem_p)
    assert ids == [0, 1, 3, 4, 5, 6, 7]
    assert {int(elem_p[e]) for e in ids} == {1, 2, 3, 4}
    assert bench.oracle_check_elements(n_elem=4096) == [0, 1365, 2730, 4095]
    assert bench.oracle_check_elements(n_elem=1) == [0]


def test_hex_traffic_table_covers_the_autotuned_dominant_kernels():
    """The hex line's roofline traffic comes from ncu captures per (kernel, dim, p,
    panel width): the FP64 element-block pair (sum-factorised volume + face terms)
    and k_elim at both panel widths of hex p = 2; per-element bytes of the right
    order (the 1.32 MB bordered matrix is read and written at least once)."""
    t = bench.DRAM_BYTES_PER_ELEMENT
    for key in (("elim", 3, 2, 16), ("elim", 3, 2, 8), ("blocks_sf", 3, 2, 0)):
        assert key in t and 1e6 < t[key] < 1e8, key
    assert t[("elim", 3, 2, 8)] > t[("elim", 3, 2, 16)]      # narrower panels re-read the trailing matrix more
