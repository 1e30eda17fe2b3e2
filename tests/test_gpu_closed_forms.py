"""The GPU tracer on hand-built scenes whose visibility has a closed form
(Eq. 13-15 with Sigma^-1; alpha = o exp(-m^2/2) at the peak): head-on and
offset hits of an isotropic Gaussian, products of k identical Gaussians on
a ray, the snap below T_min, a Gaussian behind the origin, the 3-sigma and
1/255 cut-offs, axis-aligned and rotated anisotropic Gaussians and a ray
that meets nothing; every traversal strategy.  These values come from the
formulas, not from the oracle."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
TOL = 1e-6
S2 = math.sqrt(0.5)


def _scene():
    """Cases sit 10 apart along x (the one met by a ray along x sits off the
    other cases' line), so each ray meets only its own case."""
    g = []  # (mean, scale, quat, opacity); scales and offsets are binary fractions
    iso = (0.125, 0.125, 0.125)
    ident = (1.0, 0.0, 0.0, 0.0)
    g.append(((0, 0, 0), iso, ident, 0.6))                          # 0 head-on
    g.append(((10, 0, 0), iso, ident, 0.6))                         # 1 offset
    g += [((20, 0, z), iso, ident, 0.5) for z in range(1, 6)]       # 2 five on the ray
    g += [((30, 0, z), iso, ident, 0.5) for z in range(1, 15)]      # 3 fourteen: T < T_min
    g.append(((40, 0, -1), iso, ident, 0.9))                        # 4 behind the origin
    g.append(((50, 0, 0), iso, ident, 0.6))                         # 5 3-sigma cut-off
    g.append(((60, 0, 0), iso, ident, 0.003))                       # 6 below 1/255
    g.append(((70, 0, 0), (0.125, 0.25, 0.0625), ident, 0.7))       # 7 anisotropic
    g.append(((90, 50, 0), (0.125, 0.25, 0.0625), (S2, 0, 0, S2), 0.7))  # 9 rotated 90 deg about z
    mean, scale, quat, opac = (np.array([x[i] for x in g], np.float32) for i in range(4))
    return mean, scale, quat, opac


def _rays():
    """(origin, direction, expected T in float64)."""
    a = lambda m2, o: o * math.exp(-0.5 * m2)
    return [
        ((0, 0, -1), (0, 0, 1), 1 - 0.6),
        ((10.1875, 0, -1), (0, 0, 1), 1 - a(2.25, 0.6)),      # m = 1.5
        ((20, 0, 0), (0, 0, 1), 0.5 ** 5),
        ((30, 0, 0), (0, 0, 1), 0.0),                   # 0.5^14 = 6.1e-5 < 1e-4: snapped
        ((40, 0, 0), (0, 0, 1), 1.0),                   # t* < 0
        ((50.3828125, 0, -1), (0, 0, 1), 1.0),          # m = 3.0625 > 3
        ((50.3671875, 0, -1), (0, 0, 1), 1 - a(2.9375 ** 2, 0.6)),  # m = 2.9375, alpha = 0.008 > 1/255
        ((60, 0, -1), (0, 0, 1), 1.0),                  # alpha = 0.003 < 1/255
        ((69, 0.125, 0.03125), (1, 0, 0), 1 - a(0.25 + 0.25, 0.7)),
        ((89, 50.125, 0.03125), (1, 0, 0), 1 - a(1.0 + 0.25, 0.7)),  # world x/y scales swapped
        ((80, 0, 0), (0, 0, 1), 1.0),                   # nothing there
        ((20, 0, 6), (0, 0, -1), 0.5 ** 5),             # the chain from the other end
        ((0, 0, 1), (0, 0, -1), 1 - 0.6),
    ]


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 6])
def test_closed_forms_explicit_rays(kernel):
    from paper_2311_16043_gb300 import rt
    mean, scale, quat, opac = (torch.from_numpy(x).cuda() for x in _scene())
    bvh = rt.rt_build_bvh(mean, scale, quat, opac)
    rays = _rays()
    ro = torch.tensor([r[0] for r in rays], dtype=torch.float32).cuda()
    rd = torch.tensor([r[1] for r in rays], dtype=torch.float32).cuda()
    want = np.array([r[2] for r in rays])
    rs = rt.rayspec(rt.RT_RAYS_EXPLICIT, ray_o=ro, ray_d=rd)
    T = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=kernel))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    got = T.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=0, atol=TOL)


@pytest.mark.parametrize("kernel", [0, 1, 2, 3, 4, 5, 6])
def test_closed_form_direction_set(kernel):
    """Two isotropic Gaussians 1 apart on x; the implicit rays of each along
    +x, -x and +y (origin offset 1e-4 along the ray, source skipped): the
    ray toward the other Gaussian passes 1e-4 from nothing but its centre
    line, so T = 1 - o_other; the others meet nothing."""
    from paper_2311_16043_gb300 import rt
    oA, oB = 0.3, 0.8
    mean = torch.tensor([[0, 0, 0], [1, 0, 0]], dtype=torch.float32).cuda()
    scale = torch.full((2, 3), 0.0625, dtype=torch.float32).cuda()
    quat = torch.tensor([[1, 0, 0, 0], [1, 0, 0, 0]], dtype=torch.float32).cuda()
    opac = torch.tensor([oA, oB], dtype=torch.float32).cuda()
    bvh = rt.rt_build_bvh(mean, scale, quat, opac)
    dirs = torch.tensor([[1, 0, 0], [-1, 0, 0], [0, 1, 0]], dtype=torch.float32).cuda()
    T = rt.rt_trace_visibility(bvh, rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs), opts=rt.trace_opts(kernel=kernel))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    want = np.array([[1 - oB, 1, 1], [1, 1 - oA, 1]])
    np.testing.assert_allclose(T.cpu().numpy().reshape(2, 3).astype(np.float64), want, rtol=0, atol=TOL)
