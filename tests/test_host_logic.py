"""Host-side logic that needs no GPU: how the learned batch groups sequences
for the seed network."""
from paper_1002_1168_gb300.seedtrain import chunk_plan

QCIF, CIF = (144, 176), (288, 352)


def _shape(F, size, vops):
    return (F, size[0], size[1], vops)


def test_chunks_keep_sizes_apart_and_the_callers_order():
    shapes = [_shape(10, CIF, 2), _shape(10, QCIF, 1), _shape(8, CIF, 3), _shape(10, QCIF, 4)]
    plan = chunk_plan(shapes, max_cells=10 ** 9)
    assert [(H, W) for H, W, *_ in plan] == [CIF, QCIF]  # sizes in order of first appearance
    (_, _, cif, n_cif, v_cif), (_, _, qcif, n_qcif, v_qcif) = plan
    assert cif == [(0, 0, 9), (2, 9, 7)] and n_cif == 16 and v_cif == 3
    assert qcif == [(1, 0, 9), (3, 9, 9)] and n_qcif == 18 and v_qcif == 4


def test_chunks_respect_the_network_capacity():
    cells = (288 // 4) * (352 // 4)
    shapes = [_shape(11, CIF, 1)] * 5  # 10 pairs each
    plan = chunk_plan(shapes, max_cells=25 * cells)  # room for 25 pairs: two sequences per chunk
    assert [[i for i, _, _ in m] for _, _, m, _, _ in plan] == [[0, 1], [2, 3], [4]]
    assert all(n * cells <= 25 * cells for *_, n, _ in plan)
    # offsets are contiguous inside a chunk
    for _, _, members, n, _ in plan:
        assert [off for _, off, _ in members] == [sum(P for _, _, P in members[:k]) for k in range(len(members))]
        assert n == sum(P for _, _, P in members)


def test_a_sequence_larger_than_the_network_gets_its_own_chunk():
    cells = (288 // 4) * (352 // 4)
    plan = chunk_plan([_shape(30, CIF, 1), _shape(3, CIF, 1)], max_cells=5 * cells)
    assert [[i for i, _, _ in m] for _, _, m, _, _ in plan] == [[0], [1]]


def test_reference_distance_sets_the_pair_count():
    plan = chunk_plan([_shape(10, CIF, 1), _shape(6, CIF, 2)], max_cells=10 ** 9, ref_distance=2)
    (_, _, members, n, v), = plan
    assert members == [(0, 0, 8), (1, 8, 4)] and n == 12 and v == 2
