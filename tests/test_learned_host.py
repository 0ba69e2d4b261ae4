"""Host logic of the learned-guess training set (no GPU): the sampled
elements whose exact diagonal becomes the preconditioner target."""
import numpy as np

from paper_2509_14157_gb300 import learned


def test_sample_elements_inside_sector_top_half_and_seeded():
    rng = np.random.default_rng(0)
    r2 = np.zeros(500)
    inside = np.sort(rng.choice(500, 180, replace=False))  # the spin sector
    r2[inside] = rng.uniform(1e-9, 1.0, inside.size)
    pick = learned.sample_elements(r2, 40, np.random.default_rng(7))
    assert pick.size == 40 and np.unique(pick).size == 40
    assert np.all(np.isin(pick, inside))
    top = inside[np.argsort(-r2[inside])[:20]]
    assert np.all(np.isin(top, pick))  # the 20 most important elements are always taken
    again = learned.sample_elements(r2, 40, np.random.default_rng(7))
    assert np.array_equal(pick, again)
    other = learned.sample_elements(r2, 40, np.random.default_rng(8))
    assert not np.array_equal(pick, other)


def test_sample_elements_small_sector_takes_all():
    r2 = np.zeros(50)
    r2[[3, 9, 17]] = [0.5, 1e-12, 0.1]
    assert np.array_equal(learned.sample_elements(r2, 10, np.random.default_rng(0)), [3, 9, 17])
    assert learned.sample_elements(np.zeros(20), 4, np.random.default_rng(0)).size == 0
