"""The float-pair helpers of the FP64 kernels (kg_pair.cuh), compiled for the host
with g++ and checked against long double arithmetic on seeded random inputs:
split of a double, pair -> double conversion, exact float -> double, pair
reciprocal and pair log1p; and that a chain started with acc_prod holds exactly
what acc_fma on a zero accumulator gives."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_13204_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

BOUNDS = {
    "split_f64": 2.0 ** -46,
    "pair_to_double_fast": 2.0 ** -53,
    "f32_to_f64_int": 0.0,
    "pair_recip": 2.0 ** -45,
    "pair_log1p": 2.0 ** -44,
    "pair_log1p_t": 2.0 ** -46,
    "acc_prod_vs_acc_fma": 0.0,
}


@pytest.fixture(scope="module")
def errors(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("pair") / "pair_host_check")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pair_host_check.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CUDA_INC, "-I", CSRC,
                    src, "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


@pytest.mark.parametrize("name", sorted(BOUNDS))
def test_pair_helper_error_bound(errors, name):
    assert errors[name] <= BOUNDS[name], (name, errors[name])
