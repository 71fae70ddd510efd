"""Binary 3-D volumes (every voxel 0 or 1) take the bit-sliced extraction path; other
3-D volumes of the same batch take the general 8-bit kernel.  Tables, chi, ECT and Radon
must be bit-exact against the CPU oracle whichever path built them, in mixed batches,
for rows of any length (32-voxel words with a partial last word), for constant volumes,
and for a volume of 0 / 2 voxels (two-valued but not binary: the general path).
"""
import numpy as np
import pytest

import oracle as O
from paper_2405_02256_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02256_gb300 import binding
    binding.load()
    return binding


def _check(tabs, b, img):
    ref = O.critical_tables(img)
    for o in range(8):
        idx, val = tabs.table(b, o, 0)
        np.testing.assert_array_equal(idx, ref.lower_idx[o])
        np.testing.assert_array_equal(val, ref.lower_val[o])
        assert tabs.info(b, o)[2] == ref.chi
    for r in range(4):
        idx, val = tabs.table(b, r, 1)
        np.testing.assert_array_equal(idx, ref.delta_idx[r])
        np.testing.assert_array_equal(val, ref.delta_val[r])
    return ref


def _mixed():
    return [
        synth.grf((12, 17, 33), 3.0, seed=500, binary=True),       # 33 voxels a row: a 1-bit last word
        synth.grf((9, 30, 100), 4.0, seed=501),                    # grey: general path
        synth.bernoulli((7, 8, 64), 0.5, seed=502),                # two whole words a row
        np.zeros((5, 6, 40), dtype=np.uint8),                      # all zero
        np.ones((4, 5, 31), dtype=np.uint8),                       # all one
        (2 * synth.bernoulli((6, 7, 45), 0.5, seed=503)).astype(np.uint8),   # 0 / 2: not binary
        synth.bernoulli((2, 2, 2), 0.5, seed=504),
        synth.grf((20, 24, 96), 5.0, seed=505, binary=True),
    ]


def test_mixed_batch_bit_exact(tb):
    vols = _mixed()
    tabs = tb.build_critical_tables(tb.pack_images(vols))
    for b, v in enumerate(vols):
        _check(tabs, b, v)


def test_mixed_batch_unaligned_starts(tb):
    vols = _mixed()
    tabs = tb.build_critical_tables(tb.pack_images(vols, align=1))
    for b, v in enumerate(vols):
        _check(tabs, b, v)


def test_all_binary_batch(tb):
    """Every volume binary: the general kernel has nothing to do."""
    vols = [synth.grf((14, 15, 64), 4.0, seed=530 + i, binary=True) for i in range(3)]
    tabs = tb.build_critical_tables(tb.pack_images(vols))
    for b, v in enumerate(vols):
        _check(tabs, b, v)


def test_rebuild_with_new_voxels(tb):
    """The same handle rebuilt from other voxels: a binary volume turned grey and back."""
    shape = (10, 12, 70)
    a = synth.grf(shape, 3.0, seed=510, binary=True)
    g = synth.grf(shape, 3.0, seed=511)
    tabs = tb.tables_create(tb.pack_images([a]).shapes, tb.pack_images([a]).offsets)
    for vol in (a, g, a):
        tabs.build(tb.pack_images([vol]).pixels)
        tabs.sync()
        _check(tabs, 0, vol)


def test_ect_radon_on_binary_tables(tb):
    vols = [synth.grf((16, 20, 48), 4.0, seed=520, binary=True), synth.grf((10, 11, 12), 3.0, seed=521)]
    tabs = tb.build_critical_tables(tb.pack_images(vols))
    dirs = np.concatenate([synth.fibonacci_dirs(40), np.array([[0.0, 0.0, 1.0], [1.0, -0.0, 0.0]])])
    d = torch.from_numpy(dirs).cuda()
    R = synth.image_radius(3)
    e = tb.ect(tabs, d, -R, R, 37).cpu().numpy()
    r = tb.radon(tabs, d, -R, R, 37).cpu().numpy()
    for b, v in enumerate(vols):
        ref = O.critical_tables(v)
        np.testing.assert_array_equal(e[b], O.ect_grid(ref, dirs, -R, R, 37))
        np.testing.assert_array_equal(r[b], O.radon_grid(ref, dirs, -R, R, 37))


def test_captured_graph_follows_new_voxels(tb):
    """tables_build with the binary path inside a CUDA graph (its side stream is forked and
    joined within the capture): replays with new voxels, where a binary volume turns grey
    and a grey one binary, equal the eager results."""
    shape = (12, 14, 40)
    vols_a = [synth.grf(shape, 3.0, seed=540, binary=True), synth.grf(shape, 3.0, seed=541)]
    vols_b = [synth.grf(shape, 3.0, seed=542), synth.grf(shape, 3.0, seed=543, binary=True)]
    batch_a, batch_b = tb.pack_images(vols_a), tb.pack_images(vols_b)
    R = synth.image_radius(3)
    ect_dirs = torch.from_numpy(synth.fibonacci_dirs(64)).cuda()
    ht_dirs = torch.from_numpy(synth.scale_norms(synth.fibonacci_dirs(96), 9, 0.05, 1.5)).cuda()
    pipe = tb.Pipeline(batch_a.shapes, batch_a.offsets, batch_a.pixels.numel(), ect=(ect_dirs, -R, R, 48),
                       hybrid=[("fourier", ht_dirs, "fp32c")])
    pipe.pixels.copy_(batch_a.pixels)
    pipe.capture()
    for batch in (batch_a, batch_b, batch_a):
        pipe.run(batch.pixels)
        torch.cuda.synchronize()
        eager = tb.build_critical_tables(batch)
        assert torch.equal(pipe.ect_out, tb.ect(eager, ect_dirs, -R, R, 48))
        assert torch.equal(pipe.hybrid_out[0], tb.hybrid_transform(eager, "fourier", ht_dirs))
