"""Host logic of bench.py that needs no GPU: the device-code hash that decides whether a
recorded ncu traffic figure still belongs to the kernel being timed."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """
#include <cuda_runtime.h>
__device__ __align__(16) double g_table[4];
static __device__ __forceinline__ float twice(float x) { return 2.0f * x; }
__global__ void k_scale(float* y, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { y[i] = twice(y[i]); }
}
cudaError_t launch_scale(float* y, int n, cudaStream_t s) {
  k_scale<<<(n + 255) / 256, 256, 0, s>>>(y, n);
  return cudaGetLastError();
}
"""


def test_host_edits_keep_the_device_hash():
    h = bench.device_code_sha256(SRC)
    host = SRC.replace("(n + 255) / 256, 256", "(n + 127) / 128, 128")
    assert host != SRC and bench.device_code_sha256(host) == h


def test_kernel_and_device_helper_edits_change_it():
    h = bench.device_code_sha256(SRC)
    for old, new in (("if (i < n)", "if (i <= n)"), ("2.0f * x", "3.0f * x")):
        edited = SRC.replace(old, new)
        assert edited != SRC and bench.device_code_sha256(edited) != h


def test_host_description_names_the_machine():
    h = bench.host_description()
    assert h["machine"] and h["nproc"] >= 1 and set(h) == {"machine", "nproc", "cpu_model"}


def test_step_hbm_report_sums_the_current_captures():
    r = bench.step_hbm_report("bf16x3", "C2", 3, 2.74)
    assert r is not None and r["unit"] == "GB/s" and 0 < r["frac"] < 1
    per_block = sum(n * bench.traffic_for(f, name)["dram_bytes_per_launch"]
                    for f, name, n in (("propagate_tc.cu", "propagate_tc_C2", 10),
                                       ("walker_fast.cu", "overlap_fast_C2", 10),
                                       ("gemm_tc.cu", "vhs_tc_C2", 10),
                                       ("energy_tc.cu", "energy_tc_C2", 2))
                    if bench.traffic_for(f, name))
    assert r["dram_bytes_per_block"] >= per_block > 0
    assert abs(r["achieved"] - r["dram_bytes_per_block"] / 2.74e-3 / 1e9) < 1e-9 * r["achieved"]
    assert bench.step_hbm_report("fp64", "C2", None, 2.74) is None
    assert bench.step_hbm_report("bf16x3", "C3", 3, 2.74) is None
