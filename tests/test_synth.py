"""Seeded input generators: shapes, SU(3) links, even-site bookkeeping."""
import numpy as np

import odwf_synth as syn


def test_gauge_links_are_su3():
    U = syn.gauge_field((2, 2, 2, 4), 0.3, 1).reshape(-1, 3, 3)
    assert np.abs(U @ U.conj().transpose(0, 2, 1) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_torch_gauge_links_are_su3_cpu():
    U = syn.gauge_field_torch((2, 2, 4, 2), 0.25, 3, device="cpu").numpy().reshape(-1, 3, 3)
    assert np.abs(U @ U.conj().transpose(0, 2, 1) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_random_even_site_index():
    for dims, seed in [((4, 4, 4, 4), 7), ((6, 4, 2, 8), 3), ((24, 24, 24, 48), 7)]:
        site, idx = syn.random_even_site(dims, seed)
        assert sum(site) % 2 == 0
        x, y, z, t = site
        lex = ((t * dims[2] + z) * dims[1] + y) * dims[0] + x
        if np.prod(dims) <= 4096:
            assert syn.even_sites(dims)[idx] == lex
        else:
            assert lex // 2 == idx and lex % 2 == (y + z + t) % 2
