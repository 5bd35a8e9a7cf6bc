"""Measured ALU ceilings of the GPU: FP64 and FP32 FMA throughput and the
FP64 tensor-core (DMMA, mma.sync m8n8k4) rate from the probes in
libhho_probe.so (eight independent chains per thread, eight 256-thread
blocks per SM, best of several runs), printed as multiply-add lane-ops/s and
TFLOP/s (multiply-add = 2 flops).

    python -m paper_2505_15771_gb300.peaks
"""
import ctypes
import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def rates(iters=4000, reps=5):
    lib = ctypes.CDLL(os.path.join(_HERE, "libhho_probe.so"))
    out = {}
    for name, fn, it in (("fp64", "hho_probe_dfma_rate", iters), ("fp32", "hho_probe_ffma_rate", 16 * iters),
                         ("fp64_dmma", "hho_probe_dmma_rate", iters // 4)):
        f = getattr(lib, fn)
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        r = ctypes.c_double()
        if f(it, reps, ctypes.byref(r)) != 0:
            raise RuntimeError("%s failed" % fn)
        out[name] = {"fma_lane_ops_per_s": r.value, "tflops": 2.0 * r.value / 1e12}
    # DFMA and DMMA together: time per loop of the mixed probe against the
    # two halves alone (same chains, same launch)
    f = lib.hho_probe_mixed_time
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    r = ctypes.c_double()
    it = iters // 4
    if f(it, reps, ctypes.byref(r)) != 0:
        raise RuntimeError("hho_probe_mixed_time failed")
    lanes = _lanes()
    t_dfma = lanes * 8 / out["fp64"]["fma_lane_ops_per_s"]            # one loop of 8 DFMA per thread
    t_dmma = lanes / 32 * 8 * 256 / out["fp64_dmma"]["fma_lane_ops_per_s"]   # 8 m8n8k4 per warp
    out["fp64_dfma_plus_dmma"] = {"seconds_per_loop": r.value, "dfma_alone": t_dfma, "dmma_alone": t_dmma,
                                  "overlap": (t_dfma + t_dmma) / r.value,
                                  "note": "overlap 1: the two share the FP64 hardware; 2: fully concurrent"}
    return out


def _lanes():
    """Threads of the probe launch: 8 blocks of 256 per SM."""
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count * 8 * 256


if __name__ == "__main__":
    print(json.dumps(rates(), indent=1))
