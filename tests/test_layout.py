"""Host-side checks of the shared-memory layout facts the gather kernel relies on (no GPU)."""
import itertools


def test_octant_voxels_hit_distinct_bank_pairs():
    """A brick of 4 voxels is staged as a 5 x 5 x 5 box of 12 FP16 channels (24 bytes per voxel,
    rows of 5 voxels).  The Ray Index Table sorts a brick's samples by octant (a 2 x 2 x 2 block of
    cells).  For a sample in cell v, the 64-bit load u (0..2) of corner q reads 8-byte word
    3 (v + c_q) + u, and 16 lanes of a 64-bit load share 16 bank pairs.  Two samples of one octant
    conflict only if their words differ but fall in the same pair: the 8 cells of any octant map to
    8 distinct pairs, so they never do."""
    V = 5
    for ox, oy, oz in itertools.product((0, 2), repeat=3):
        cells = [(ox + dx) + V * (oy + dy) + V * V * (oz + dz) for dx, dy, dz in itertools.product((0, 1), repeat=3)]
        for q in range(8):
            c_q = (q & 1) + V * ((q >> 1) & 1) + V * V * (q >> 2)
            for u in range(3):
                pairs = [(3 * (v + c_q) + u) % 16 for v in cells]
                assert len(set(pairs)) == 8, (ox, oy, oz, q, u)


def test_octant_of_brick_matches_the_key_bits():
    """The key's octant bits are bit (log2(B) - 1) of the voxel index along x, y, z: the upper half
    of the brick along each axis."""
    for B, h in ((4, 1), (8, 2), (16, 3)):
        for i in range(3 * B):
            assert ((i >> h) & 1) == int((i % B) >= B // 2)
