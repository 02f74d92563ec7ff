"""The autotuner's candidate shapes and the serving layer's reading of its table, on the host."""
import json

import paper_1905_01348_gb300.autotune as at
import paper_1905_01348_gb300.serve as serve


def test_candidates_cover_tiles_and_group_sizes():
    c = at.candidates(16, 12)
    assert {(4, 0), (3, 0), (2, 0)} <= set(c)
    # tile 4: the largest merged round of 12 systems of 16 orbitals has 12 x 4 = 48 tiles -> 24, 12, 6
    assert {(4, 24), (4, 12), (4, 6)} <= set(c)
    assert all(t >= 0 for _, t in c)
    assert {tile for tile, _ in at.candidates(1, 3)} == {1}
    assert {tile for tile, _ in at.candidates(3, 3)} == {3, 2}


def test_serving_reads_the_table(tmp_path):
    table = {"si8-mixed": {"systems": 12, "best": {"pair_tile": 4, "tiles_per_launch": 24}, "measured": []}}
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps(table))
    assert serve.tuned_batch_shape("si8", "mixed", str(path)) == {"pair_tile": 4, "tiles_per_launch": 24}
    assert serve.tuned_batch_shape("si64", "mixed", str(path)) == {"pair_tile": 0, "tiles_per_launch": 0}
    assert serve.tuned_batch_shape("si8", "mixed", str(tmp_path / "absent.json")) == {"pair_tile": 0,
                                                                                     "tiles_per_launch": 0}
