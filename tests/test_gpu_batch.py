"""Batched tissues (daeti_batch_*): every tissue equals the same tissue advanced
alone, bit for bit, and the batch covers mixed models, sizes and stimuli."""
import numpy as np
import pytest

import inputs as I
from parity_util import act_error, ensure_lib, gpu_available, run_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp64"])
def test_batch_equals_single_tissues(precision):
    binding = ensure_lib()
    wls = I.batch_tissues(n_tissues=14, side_min=6, side_max=30, t_end=20.0)
    wls.append(I.tp06_slab_3d(9, 7, 5))                   # a 3D tissue in the same batch
    batch = binding.Batch(precision=precision, graph_steps=10)
    descs = [binding.describe_workload(w, precision=precision) for w in wls]
    for d in descs:
        batch.daeti_batch_add(d)
    for d in descs:
        d.close()
    batch.daeti_batch_prepare()
    info = batch.daeti_batch_info()
    assert info["n_tissues"] == len(wls) and info["n_nodes"] == sum(w.n_nodes for w in wls)
    batch.daeti_batch_advance(7.0)
    batch.daeti_batch_advance(20.0)
    for t, w in enumerate(wls):
        s = binding.solver_from_workload(w, precision=precision)
        s.daeti_advance(20.0)
        v, a = s.daeti_read_v(), s.daeti_read_activation()
        s.close()
        assert np.array_equal(batch.daeti_batch_read_v(t), v), t
        assert np.array_equal(batch.daeti_batch_read_activation(t), a), t
    batch.close()


def test_batch_tissue_against_oracle():
    binding = ensure_lib()
    wls = I.batch_tissues(n_tissues=4, side_min=10, side_max=16, t_end=15.0)
    batch = binding.Batch(precision="fp64")
    for w in wls:
        d = binding.describe_workload(w, precision="fp64")
        batch.daeti_batch_add(d)
        d.close()
    batch.daeti_batch_prepare()
    batch.daeti_batch_advance(15.0)
    for t, w in enumerate(wls):
        o, oa, _ = run_oracle(w, 150, 150)
        mv = 100.0 if w.model == "ms" else 1.0
        assert float(np.max(np.abs(batch.daeti_batch_read_v(t) - o[-1]))) * mv <= 0.5
        da, same, _ = act_error(batch.daeti_batch_read_activation(t), oa)
        assert same and da <= 0.1
    batch.close()


def test_batch_rejects_mixed_model_parameters():
    binding = ensure_lib()
    a = I.ms_square_2d(n=8)
    b = I.ms_square_2d(n=9)
    b.model_params = (0.3, 6.0, 120.0, 140.0, 0.13)
    batch = binding.Batch()
    for w in (a, b):
        d = binding.describe_workload(w)
        batch.daeti_batch_add(d)
        d.close()
    with pytest.raises(binding.DaetiError) as e:
        batch.daeti_batch_prepare()
    assert e.value.code == binding.EUNSUPPORTED
    batch.close()
