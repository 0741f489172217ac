"""Host logic of the ensemble autotuner's option sets (no GPU): every
combination of tile width, sweeps, relaxation factor and coarse-level sweeps
once, plus the library default without graphs as the reference point; and
the admission footprint estimate counts the Poisson guess history."""
from paper_2505_17287_gb300 import ensemble, ibm


def test_candidates_cover_the_grid_once():
    cand = ensemble.candidates()
    assert len(cand) == 4 * 2 * 2 * 2 + 1
    keys = [(o.tile_x, o.nu1, o.nu2, o.smooth_omega, o.nu_coarse, o.graph) for o in cand[:-1]]
    assert len(set(keys)) == len(keys)
    assert {k[4] for k in keys} == {0, 3} and all(k[1] == k[2] and k[5] == 1 for k in keys)
    ref, dflt = cand[-1], ibm.ibm_default_opts()
    assert ref.graph == 0 and ref.nu_coarse == dflt.nu_coarse and ref.nu2 == dflt.nu2
    d = ensemble.describe(cand[0])
    assert set(d) == {"tile_x", "nu", "nu2", "nu_coarse", "omega", "graph"}


def test_case_bytes_counts_the_guess_history():
    n = 128 ** 3
    b = ibm.ibm_case_bytes(3, 128, 128, 128, ibm.IBM_MIXED, 5120)
    assert b >= 1.25 * (8 + 16 * 8) * n
