"""Host logic of the ragged-batch autotuner (CPU): every candidate shape is one the batch
planner accepts -- its lane mapping covers the instance's frames and its voxel box holds
exactly the voxels one block of that mapping covers."""
import pytest

from paper_2604_06257_gb300 import autotune


def block_voxels(mode, frame_lanes):
    """Voxels of one batch block per lane mapping: channel lanes 8 warps x 4 voxels; frame
    lanes 8 warps x (32 / FL) lane groups x 4 voxels (2 voxels per lane pair for FL = 2);
    staged windows 7 consumer warps x (32 / FL) lane groups x 4 voxels."""
    if mode == 1:
        return 32
    if mode == 2:
        return 7 * 4 * (32 // frame_lanes)
    return 256 if frame_lanes == 2 else 8 * 4 * (32 // frame_lanes)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("F", [1, 3, 4, 5, 8, 9, 16, 17, 32, 33, 48, 64])
def test_candidates_are_valid_shapes(ndim, F):
    cands = autotune.candidates({"n_frames": F, "ndim": ndim})
    assert cands, F
    modes = {c[0] for c in cands}
    assert (1 in modes) == (F <= 4)                       # channel lanes only for short ensembles
    for mode, fl, box in cands:
        assert mode in (0, 1, 2)
        if mode == 1:
            assert fl == 0
        else:
            assert fl in ((2, 4, 8, 16) if mode == 0 else (8, 16)) and 4 * fl >= F
        assert box[0] * box[1] * box[2] == block_voxels(mode, fl), (mode, fl, box)
        if ndim == 2:
            assert box[1] == 1
    # the two-lane mapping is offered exactly where its 8 frame slots suffice
    assert any(m == 0 and fl == 2 for m, fl, _ in cands) == (F <= 8)
