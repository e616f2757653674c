"""Small, self-contained launches of each kernel family for profiling with ncu
(python -m paper_2109_04469_gb300.profile_cases fp64|ens|mlp): the FP64 particle pass on the
production workload, a 16-member ensemble step, and the surrogate network's training GEMMs."""
from __future__ import annotations

import sys


def main(mode: str) -> None:
    import torch

    from . import pic, workloads

    if mode == "fp64":  # 5 steps of the FP64 plain path, 2e6 + 2e6 superparticles
        sim = pic.Simulation(workloads.params("ccp_1pa_300v_400c", precision=pic.PIC_FP64))
        sim.step(5)
        print("status", sim.sync())
    elif mode == "ens":  # 16 scan members (2.5e5-1e6 superparticles each), 5 ensemble steps
        members = workloads.ensemble_members(16, per_run=(2.5e5, 1.0e6))
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            sims = [pic.Simulation(dict(c, precision=pic.PIC_FP32)) for c, _ in members]
            ens = pic.Ensemble(sims, [10**9] * len(sims))
            ens.configure(2048, 2, True)
            ens.step(5)
        try:
            print("status", ens.sync())
        except pic.PicError as e:  # births dropped at capacity in the fastest members
            print("status", e.code)
    elif mode == "mlp":  # 3 Adam steps of the surrogate network at batch 1024
        net = pic.Mlp(1024, seed=1)
        x = torch.randn(1024, 7, device="cuda")
        t = torch.randn(1024, 192, device="cuda")
        for _ in range(3):
            net.train_step(x, t, 1e-3, want_loss=False)
        torch.cuda.synchronize()
        print("ok")
    else:
        raise SystemExit("mode: fp64 | ens | mlp")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "")
