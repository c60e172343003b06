"""Parity at the full sizes of the 3D workloads, in the launch configuration
the benchmark times: one step of the 256^3 shock-droplet and of the
512x256x256 shock-bubble grids, perturbed so that every cell differs,
checked at sampled nodes (every face, edge and corner region, tile seams and
random interior nodes) against the oracle evaluated node by node."""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sample_nodes(nx, ny, nz, seed, n_random=3000):
    rng = np.random.default_rng(seed)
    pts = [rng.integers(0, n, n_random) for n in (nx, ny, nz)]
    xyz = list(np.stack(pts, axis=1))
    edge = lambda n: sorted({0, 1, 2, n // 2, 31, 32, 33, n - 3, n - 2, n - 1} & set(range(n)))
    for x in edge(nx):
        for y in edge(ny):
            for z in edge(nz):
                xyz.append((x, y, z))
    return np.asarray(xyz, dtype=np.int32)


def _perturbed(w, seed):
    rho, u, T = w.initial_fields()
    rho = rho * (1.0 + workloads.noise(rho.shape, seed, 0.05))
    T = T * (1.0 + workloads.noise(T.shape, seed + 1, 0.05))
    u = u + workloads.noise(u.shape, seed + 2, 0.05)
    return rho, u, T


@pytest.mark.parametrize("which,precision", [("droplet", "fp32"), ("droplet", "fp64"), ("bubble", "fp32")])
def test_one_step_at_full_size(which, precision):
    from paper_1010_4135_gb300 import sim as S
    w = workloads.shock_droplet() if which == "droplet" else workloads.shock_bubble()
    cfg = oracle.cfg_for(w)
    rho, u, T = _perturbed(w, seed=17)
    f0 = oracle.init(cfg, rho, u, T)
    del rho, u, T
    if precision == "fp32":
        f0 = f0.astype(np.float32)
    s = S.from_workload(w, precision=precision)
    s.set_f(f0)
    s.step(1)
    g = s.get_f()
    s.close()
    xyz = _sample_nodes(w.nx, w.ny, w.nz, seed=3)
    ref = oracle.step_nodes(cfg, f0.astype(np.float64) if precision == "fp32" else f0, xyz)
    got = np.stack([g[:, z, y, x] for x, y, z in xyz]).astype(np.float64)
    err = field_errors(got.T, ref.T)
    tol = 1e-12 if precision == "fp64" else 5e-6
    assert err.max() <= tol, err
