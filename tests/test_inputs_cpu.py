"""The synthetic Moana-scale workload against the scene statistics the paper
prints (Figure 1 caption), and the transcription of the paper's Table 1."""
import numpy as np

from paper_2001_02620_gb300 import inputs as I
from golden_data import moana_statistics, table1


def test_moana_generator_matches_the_papers_statistics():
    g = moana_statistics()
    n, c, terrain = I.moana_sizes(1.0)
    unique = int(n.sum()) + terrain
    instances = int(c.sum())
    instanced = int((n * c).sum()) + terrain
    # the paper prints these to three or four significant digits
    assert abs(unique - g["unique_quads"]) <= 0.0005 * g["unique_quads"]
    assert abs(instances - g["instances"]) <= 0.0005 * g["instances"]
    assert abs(instanced - g["instanced_quads"]) <= 0.005 * g["instanced_quads"]
    # heavy instancing skewed to small prototypes: mean quads per instance
    # far below the mean prototype size
    assert instanced / instances < 0.1 * unique / len(n)


def test_generator_constants_are_the_papers():
    g = moana_statistics()
    assert I.MOANA_QUADS == g["unique_quads"]
    assert I.MOANA_INSTANCES == g["instances"]
    assert I.MOANA_INSTANCED_QUADS == g["instanced_quads"]


def test_table1_columns_sum_to_one_hundred_percent():
    t = table1()
    cols = np.array(list(t.values())).sum(axis=0)
    np.testing.assert_allclose(cols, 100.0, atol=0.02)
    assert min(t["traversal_and_intersection"]) == 67.28


def test_heat_map_writer(tmp_path):
    import torch
    from paper_2001_02620_gb300 import api
    c = torch.arange(12, dtype=torch.float32).reshape(3, 4)
    p = str(tmp_path / "cost.ppm")
    scale = api.save_heat_map(c, p, scale=11.0)
    data = open(p, "rb").read()
    assert data.startswith(b"P6\n4 3\n255\n") and len(data) == len(b"P6\n4 3\n255\n") + 36
    px = np.frombuffer(data[-36:], dtype=np.uint8).reshape(3, 4, 3)
    assert scale == 11.0 and px[0, 0].tolist() == [0, 0, 0] and px[2, 3].tolist() == [255, 255, 255]
