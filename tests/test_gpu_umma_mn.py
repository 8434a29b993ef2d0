"""The MN-major operand path of tcgen05.mma (sml_debug_umma_mn), the operand layout of the
weight-gradient contraction of the tensor-core training kernels (its K runs over pixels):
one product D = A B^T against a float64 matmul of the same bf16 values, with B's
descriptor started several lines into its planes (the tap shift along the pixels)."""
import numpy as np
import pytest
import torch

import paper_2410_02314_gb300 as sml

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def bf16_round(x):
    return torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def mn_image(mat, plane_bytes, nplanes, shift=0):
    """Shared-memory image of a (rows x K) bf16 matrix as MN-major 32-byte-swizzled planes:
    plane g holds rows 16g..16g+15, line `shift + k` holds column k (32 bytes: the 16 rows),
    and the 16-byte chunks are permuted by the 32-byte swizzle (chunk bit 0 ^= chunk bit 3)."""
    R, K = mat.shape
    lines = plane_bytes // 32
    assert shift + K <= lines and R <= 16 * nplanes
    bits = torch.from_numpy(mat.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    img = np.zeros((nplanes, lines, 16), dtype=np.uint16)
    for r in range(R):
        img[r // 16, shift : shift + K, r % 16] = bits[r]
    chunks = img.reshape(-1, 8)  # 16-byte chunks
    idx = np.arange(chunks.shape[0])
    phys = np.empty_like(chunks)
    phys[idx ^ ((idx >> 3) & 1)] = chunks
    return phys.reshape(-1).view(np.uint8)


def run(A, B, M, N, K, a_plane, b_plane, shift):
    a_img = mn_image(A, a_plane, M // 16)
    b_img = mn_image(B, b_plane, N // 16, shift)
    pad = lambda x: np.concatenate([x, np.zeros((-x.size) % 1024, np.uint8)])
    a_img, b_img = pad(a_img), pad(b_img)
    da, db = torch.from_numpy(a_img).cuda(), torch.from_numpy(b_img).cuda()
    dd = torch.zeros((128, N), dtype=torch.float32, device="cuda")
    code = sml.lib().sml_debug_umma_mn(da.data_ptr(), db.data_ptr(), dd.data_ptr(), M, N, K, a_img.size, b_img.size,
                                       a_plane, b_plane, shift, torch.cuda.current_stream().cuda_stream)
    assert code == sml.SML_OK
    return dd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("rows,N,K,shift", [(48, 48, 32, 0), (48, 48, 64, 5), (48, 16, 32, 3), (128, 144, 48, 17)])
def test_mn_major_m128(rows, N, K, shift):
    """M = 128 (rows beyond `rows` zero, as the 48 output channels of the weight gradient pad
    to 128): D[m, n] = sum_k A[m, k] B[n, k] in TMEM lane m."""
    rng = np.random.default_rng(rows + N + K + shift)
    A = np.zeros((128, K))
    A[:rows] = bf16_round(rng.uniform(-1, 1, (rows, K)))
    B = bf16_round(rng.uniform(-1, 1, (N, K)))
    lines = ((shift + K + 7) // 8) * 8
    got = run(A, B, 128, N, K, 128 * 32, max(256, lines * 32), shift)
    want = A @ B.T
    assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max())
