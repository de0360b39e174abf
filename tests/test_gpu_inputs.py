"""The GPU twin of the seeded quadruple generator is bit-identical to the numpy one."""
import numpy as np
import pytest

import coulomb_inputs as ci
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("R", [4, 13, 63])
@pytest.mark.parametrize("stream", [ci.STREAM_CLEAN, ci.STREAM_PLANTED, ci.STREAM_UNIFORM])
def test_device_generator_matches_numpy(R, stream):
    import torch
    dev = need_gpu()
    host = ci.quads_uniform if stream == ci.STREAM_UNIFORM else ci.quads
    for start, n in ((0, 5000), (987654321, 3001)):
        out = torch.empty((n, 4), dtype=torch.int32, device=dev)
        ci.quads_device(R, start, n, out, stream=stream)
        assert np.array_equal(out.cpu().numpy(), host(R, start, n, stream=stream))
