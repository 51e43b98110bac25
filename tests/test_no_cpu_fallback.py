"""Every public compute call of the binding refuses host data: there is no CPU fallback, so on a
machine without a GPU (or with host tensors) each call raises instead of computing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1204_5041_gb300 as isw  # noqa: E402


def _h(*shape, dtype=torch.float64):
    return torch.zeros(*shape, dtype=dtype)


CALLS = {
    "hp_pix2vec_ring": lambda: isw.hp_pix2vec_ring(4, pix=_h(3, dtype=torch.int64)),
    "hp_vec2pix_ring": lambda: isw.hp_vec2pix_ring(4, _h(3, 5)),
    "lightcone_intersect": lambda: isw.lightcone_intersect(isw.LINEAR, _h(10, 5)),
    "lightcone_intersect_shells": lambda: isw.lightcone_intersect_shells(_h(10, 5), [0, 5], [0.5], [0]),
    "isw_map": lambda: isw.isw_map(4, _h(10, 5)),
    "isw_map_adjoint": lambda: isw.isw_map_adjoint(4, _h(10, 5), _h(192)),
    "isw_map_batched": lambda: isw.isw_map_batched(4, _h(10, 5), [0, 5], [0.5], [0]),
    "lightcone_adjoint": lambda: isw.lightcone_adjoint(isw.LINEAR, _h(10, 5), _h(5), _h(6, 5)),
    "box_place": lambda: isw.box_place(_h(10, 5), [0, 5], [0], _h(1, 12)),
    "cone_cut": lambda: isw.cone_cut(_h(10, 5), [0, 5], 1, _h(1, dtype=torch.int64), _h(1), _h(1)),
    "isw_map_patch": lambda: isw.isw_map_patch(np.eye(3), 4, 0.1, _h(10, 5)),
    "isw_map_cl": lambda: isw.isw_map_cl(4, _h(192), 8),
}


@pytest.mark.parametrize("name", sorted(CALLS))
def test_host_data_is_refused(name):
    with pytest.raises(Exception):
        CALLS[name]()
