"""Small, self-contained GPU cases for profiling single kernels with ncu.

    python -m paper_1308_5426_gb300.profile_case <case>

cases:
  chains_fp64   8 chains L=1024 q=5 R=64, FP64 fields (shared-memory sweep kernel), 4 sweeps
  chains_fp32   the same chains in FP32 (register-resident sweep kernel), 4 sweeps
  chains_fx64   the same chains with 64-bit fixed-point fields (register-resident sweep kernel), 4 sweeps
  chains_fx64_memory  the same FX64 chains with the fields in shared memory, 4 sweeps
  precision_fp32  L=4096 q=8 R=128, FP32 (register-resident sweep), 3 sweeps
  precision_fp64  L=4096 q=8 R=128, FP64 fields shared by two-CTA clusters, 3 sweeps
  precision_fx64  L=4096 q=8 R=128, FX64 fields shared by two-CTA clusters, 3 sweeps
  precision_fp64_eq  the same FP64 job with its automatic cluster size (four CTAs on 152 SMs):
                200 sweeps + exchanges to equilibrate, then 2 more
  rebuild_fp32  L=4096 q=8 R=128, FP32: 3 tensor-core field rebuilds + measurements
  rebuild_fp32_long  L=16384 q=5 R=64, FP32: 3 tensor-core field rebuilds + measurements
  long_fp32     one job L=16384 q=5 R=64, FP32, fields in global memory (memory kernel), 3 sweeps
  long_fp32_cluster  the same job with its fields shared by a two-CTA cluster, 3 sweeps
  long_fp32_rcluster  the same job with its fields in the registers of a four-CTA cluster, 3 sweeps
  hot_fp32_rcluster   L=16384 q=5, four slots at T = Jtot (acceptance 0.86), FP32 fields in the
                      registers of four-CTA clusters; 10 sweeps to equilibrate, then 2
Each case builds its jobs, runs, synchronises and exits 0; inputs are the
seeded workloads of paper_1308_5426_gb300.workloads.
"""
import sys


def main(argv):
    import paper_1308_5426_gb300 as plr
    from paper_1308_5426_gb300 import workloads

    case = argv[1] if len(argv) > 1 else ""
    variant = "auto"
    if case in ("chains_fp64", "chains_fp32", "chains_fx64"):
        specs, prec, nsw = workloads.chains_jobs(), case[-4:], 4
    elif case == "chains_fx64_memory":
        specs, prec, nsw, variant = workloads.chains_jobs(), "fx64", 4, "memory"
    elif case in ("precision_fp32", "precision_fp64", "precision_fx64"):
        prec = case[-4:]
        specs, nsw = [workloads.precision_job(prec)], 3
        if prec != "fp32":
            variant = "cluster"
    elif case == "precision_fp64_eq":
        s = workloads.precision_job("fp64")
        j = plr.Job(s.L, s.q, s.sigma, s.ratios * plr.jtot(s.L, s.sigma), s.seed, precision="fp64")
        for _ in range(202):
            j.sweep(1)
            j.exchange()
        j.sync()
        print("ok", case, j.sweep_info()["cluster"])
        return 0
    elif case in ("long_fp32", "long_fp32_cluster", "long_fp32_rcluster"):
        from paper_1308_5426_gb300.workloads import geometric_ratios
        L, q = 16384, 5
        v = {"long_fp32": "memory", "long_fp32_cluster": "cluster", "long_fp32_rcluster": "rcluster"}[case]
        j = plr.Job(L, q, 0.4, geometric_ratios(64, 0.05, 1.0) * plr.jtot(L, 0.4), 3, precision="fp32",
                    recompute_every=0, sweep_variant=v)
        for _ in range(3):
            j.sweep(1)
            j.exchange()
        j.sync()
        print("ok", case)
        return 0
    elif case == "hot_fp32_rcluster":
        import numpy as np
        L = 16384
        j = plr.Job(L, 5, 0.4, np.full(4, plr.jtot(L, 0.4)), 3, precision="fp32", recompute_every=0,
                    sweep_variant="rcluster")
        for _ in range(12):
            j.sweep(1)
        j.sync()
        print("ok", case)
        return 0
    elif case in ("rebuild_fp32", "rebuild_fp32_long"):
        s = workloads.precision_job("fp32")
        if case == "rebuild_fp32_long":
            s = workloads.JobSpec(L=16384, q=5, sigma=0.4, ratios=workloads.geometric_ratios(64, 0.05, 1.0), seed=3,
                                  sweeps=1, precision="fp32")
        j = plr.Job(s.L, s.q, s.sigma, s.ratios * plr.jtot(s.L, s.sigma), s.seed, precision="fp32",
                    recompute_every=0)
        j.sweep(1)
        for _ in range(3):
            j.fields_recompute()
            j.measure()
        j.sync()
        print("ok", case)
        return 0
    else:
        print(__doc__)
        return 2
    jobs = [plr.Job(s.L, s.q, s.sigma, s.ratios * plr.jtot(s.L, s.sigma), s.seed, precision=prec,
                    recompute_every=0, sweep_variant=variant) for s in specs]
    b = plr.Batch(jobs)
    for _ in range(nsw):
        b.sweep(1)
        b.exchange()
    b.sync()
    print("ok", case)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
