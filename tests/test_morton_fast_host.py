"""Host check of the error bound behind the Morton kernel's division-free 10-bit quantisation
(Sec. 2.1, Morton codes scaled by the scene box).

The kernel computes f = fl(x * fl(2^10 fl(1 / ext))) and accepts floor(f) when f lies at least
2^-11 inside a cell [c, c + 1) with 0 <= c <= 1023; otherwise it divides exactly.  The claim is
|f - 2^10 fl(x / ext)| <= 1.9e-4 for 0 <= x <= ext, so an accepted cell is the exact one.  Here
the same FP32 operations run in numpy (IEEE single precision, correctly rounded, no fused
multiply-add) over many extents and offsets, including values packed against cell edges."""
import numpy as np

EPS = np.float32(2.0 ** -11)


def _check(ext: np.float32, x: np.ndarray):
    x = x.astype(np.float32)
    u = (x / ext).astype(np.float32)                         # the exact form's fl(x / ext)
    rs = np.float32(np.float32(1.0) / ext) * np.float32(1024.0)
    f = (x * rs).astype(np.float32)
    exact_scaled = u.astype(np.float64) * 1024.0             # 2^10 u, exact in float64
    assert np.all(np.abs(f.astype(np.float64) - exact_scaled) <= 1.9e-4)
    cell = np.floor(f)
    fr = (f - cell).astype(np.float32)
    ok = (fr >= EPS) & (fr <= np.float32(1) - EPS) & (cell >= 0) & (cell <= 1023)
    q_exact = np.minimum(np.floor(np.clip(u, 0, 1).astype(np.float32) * np.float32(1024.0)), 1023)
    assert np.array_equal(cell[ok], q_exact[ok])
    return ok.mean()


def test_division_free_quantisation_matches_the_division():
    rng = np.random.default_rng(11807)
    exts = [np.float32(v) for v in (1.0, 3.0, 0.7, 1e-3, 2.5e-20, 7.3e19, 0.0062035, 255.0, 1.1)]
    exts += [np.float32(v) for v in 10.0 ** rng.uniform(-30, 30, 12)]
    accepted = []
    for ext in exts:
        x = rng.uniform(0, 1, 400_000) * np.float64(ext)
        j = rng.integers(0, 1025, 200_000)
        edge = (j * np.float64(ext) / 1024).astype(np.float32)  # on the cell edges ...
        near = np.concatenate([np.nextafter(edge, np.float32(np.inf)), np.nextafter(edge, np.float32(0)), edge])
        margin = (j + rng.choice([2 ** -11, 1 - 2 ** -11, 2 ** -12, 1.5 * 2 ** -11], j.size)) * np.float64(ext) / 1024
        xs = np.clip(np.concatenate([x, near, margin]).astype(np.float32), np.float32(0), ext)
        _check(ext, xs)
        accepted.append(_check(ext, np.clip(x.astype(np.float32), np.float32(0), ext)))
    # uniform coordinates take the multiply except within the margin of an edge (about 2^-10)
    assert min(accepted) > 0.99
