"""Forward and backward cases that take every shared-memory path of the
deposit and the adjoint (centre samples and bin means on the fast path, the
per-bin and global paths, BF16 templates, a split heavy spaxel), run with
one build of the library and saved for comparison with another.

    python tests/_debug_cases.py debug|release OUT.npz

Run as a separate process by tests/test_gpu_debug_build.py: a process loads
one build of the library only."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)


def _cases():
    from paper_2412_08265_gb300 import synth
    out = []
    base = synth.mid_galaxy(n=60_000, seed=23)
    tel = synth.Telescope(nx=32, ny=32, spaxel_size=0.3, n_lambda=3721, lambda0=4750.0, dlambda=1.25)
    out.append(("centre_f32", base.ssp, tel, base.particles, "f32"))
    out.append(("centre_bf16", base.ssp, tel, base.particles, "bf16"))
    bm = synth.Telescope(nx=20, ny=20, spaxel_size=0.5, n_lambda=3721, lambda0=4750.0, dlambda=1.25,
                         flux_scale=2e-3, resample=1)
    out.append(("bin_means", base.ssp, bm, base.particles, "f32"))
    out.append(("bin_means_general", base.ssp,
                synth.Telescope(nx=20, ny=20, spaxel_size=0.5, n_lambda=1583, lambda0=4760.0, dlambda=2.9,
                                flux_scale=2e-3, resample=1), base.particles, "f32"))
    hv = base.particles.subset(np.arange(base.particles.n))
    hv.v_los = hv.v_los.copy()
    hv.v_los[::7] = np.float32(4000.0)
    hv.v_los[3::7] = np.float32(-3500.0)
    out.append(("high_velocity", base.ssp, tel, hv, "f32"))
    heavy = synth.mid_galaxy(n=5000, seed=24).particles
    heavy.x = np.full_like(heavy.x, 0.05)
    heavy.y = np.full_like(heavy.y, 0.05)
    out.append(("split_heavy", base.ssp, synth.Telescope(nx=5, ny=5, spaxel_size=0.3, n_lambda=3721,
                                                         lambda0=4750.0, dlambda=1.25), heavy, "f32"))
    return out


def run(debug: bool, path: str):
    import torch
    from paper_2412_08265_gb300 import build as B
    from paper_2412_08265_gb300 import capi
    capi.load(B.build(debug=debug))
    from paper_2412_08265_gb300.model import CubeModel
    torch.cuda.set_device(0)
    res = {}
    for name, ssp, tel, p, dtype in _cases():
        model = CubeModel(ssp, tel, dtype, max_particles=p.n)
        cube = model.forward(p)
        st = model.stats()
        rng = np.random.default_rng(5)
        G = torch.from_numpy(rng.standard_normal(model.cube_shape).astype(np.float32)).cuda()
        grads = model.backward(G)[:4]
        torch.cuda.synchronize()
        res[f"{name}/cube"] = cube.cpu().numpy()
        for k, g in zip(("dm", "dage", "dZ", "dv"), grads):
            res[f"{name}/{k}"] = g.cpu().numpy()
        res[f"{name}/err"] = np.array([st["device_error"]], dtype=np.int64)
        res[f"{name}/slow"] = np.array([st["slow_particle_tiles"]], dtype=np.int64)
        model.close()
    np.savez(path, **res)


if __name__ == "__main__":
    run(sys.argv[1] == "debug", sys.argv[2])
