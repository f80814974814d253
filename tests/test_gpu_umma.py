"""Unit probes of the tcgen05 primitives (descriptors, TMEM, mbarrier) that
the tensor-core forward kernels use, against float32 matmul / convolution
of the same bf16 values."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "cuda", "umma_probe.cu")
OUT = os.path.join(ROOT, "paper_2307_09063_gb300", "_build", "libumma_probe.so")


@pytest.fixture(scope="module")
def probe():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-o", OUT, SRC], check=True)
    L = ctypes.CDLL(OUT)
    L.probe_gemm.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.probe_conv.argtypes = [ctypes.c_void_p] * 4
    return L


state = {"gemm_ok": False}


@pytest.mark.parametrize("N,K", [(16, 16), (32, 64), (64, 32)])
def test_umma_gemm(probe, N, K):
    g = torch.Generator().manual_seed(N * 100 + K)
    A = torch.randn(128, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    D = torch.zeros(128, N, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ad, Bd = A.cuda(), B.cuda()
    assert probe.probe_gemm(Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), N, K, st.data_ptr()) == 0
    assert int(st.item()) == 0
    ref = A.float() @ B.float().T
    assert torch.allclose(D.cpu(), ref, rtol=1e-5, atol=1e-4), (D.cpu() - ref).abs().max()
    state["gemm_ok"] = True


def test_umma_shifted_conv(probe):
    if not state["gemm_ok"]:
        pytest.skip("descriptor layout not confirmed by the GEMM probe")
    Wp, R = 16, 10
    g = torch.Generator().manual_seed(7)
    img = torch.zeros(R, Wp, 16)
    img[1:9, 1:15] = torch.randn(8, 14, 16, generator=g)
    X = img.to(torch.bfloat16)
    Wt = torch.randn(9, 32, 16, generator=g).to(torch.bfloat16)  # [tap][cout][cin]
    D = torch.zeros(128, 32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Xd, Wd = X.reshape(-1, 16).contiguous().cuda(), Wt.contiguous().cuda()
    assert probe.probe_conv(Xd.data_ptr(), Wd.data_ptr(), D.data_ptr(), st.data_ptr()) == 0
    assert int(st.item()) == 0
    flat = torch.zeros(320, 16)
    flat[:R * Wp] = X.float().reshape(-1, 16)
    ref = torch.zeros(128, 32)
    for t in range(9):
        sh = (t // 3 - 1) * Wp + (t % 3 - 1)
        ref += flat[Wp + 1 + sh: Wp + 1 + sh + 128] @ Wt[t].float().T
    assert torch.allclose(D.cpu(), ref, rtol=1e-5, atol=1e-3), (D.cpu() - ref).abs().max()
