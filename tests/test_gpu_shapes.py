"""The binding rejects wrongly shaped buffers before anything reaches the
library: each call below raises ValueError (TypeError for a wrong dtype) and
launches no kernel (the library's own launch counter is unchanged). A wrongly
sized buffer passed on as a raw pointer would otherwise be read or written
out of bounds."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_09313_gb300 as lib
    return lib


def z(*shape, dtype=torch.float32):
    return torch.zeros(shape, dtype=dtype, device="cuda")


def cases(nmf):
    k, nrhs = 10, 32
    G, B = z(k, k, dtype=torch.float64), z(nrhs, k)
    yield "G not k x k", lambda: nmf.nmf_nls_bpp(z(k + 1, k + 1, dtype=torch.float64), B)
    yield "passive_in rows", lambda: nmf.nmf_nls_bpp(G, B, passive_in=z(nrhs - 1, 1,
                                                                        dtype=torch.int64))
    yield "passive_in words", lambda: nmf.nmf_nls_bpp(G, B, passive_in=z(nrhs, 2,
                                                                         dtype=torch.int64))
    yield "noalloc G", lambda: nmf.nmf_nls_bpp_noalloc(z(k - 1, k - 1, dtype=torch.float64), B)
    yield "tune G", lambda: nmf.nmf_nls_bpp_tune(z(k, k + 1, dtype=torch.float64), B)
    A = z(40, 30)
    yield "mm F rows", lambda: nmf.nmf_mm_dense(A, z(40, 5), False)
    yield "mm F rows (trans)", lambda: nmf.nmf_mm_dense(A, z(30, 5), True)
    yield "mm out shape", lambda: nmf.nmf_mm_dense(A, z(30, 5), False, out=z(40, 6))
    yield "mm out dtype", lambda: nmf.nmf_mm_dense(A, z(30, 5), False,
                                                   out=z(40, 5, dtype=torch.float64))
    yield "mm out strided", lambda: nmf.nmf_mm_dense(A, z(30, 5), False, out=z(40, 10)[:, :5])
    rp = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    ci = torch.tensor([0, 3], dtype=torch.int32, device="cuda")
    vals = z(2)
    yield "csr F rows", lambda: nmf.nmf_mm_csr(rp, ci, vals, 4, z(5, 3))
    yield "csr vals length", lambda: nmf.nmf_mm_csr(rp, ci, z(3), 4, z(4, 3))
    yield "csr transpose rowptr", lambda: nmf.nmf_csr_transpose(rp, ci, vals, 3, 4)
    yield "init Ht0 columns", lambda: nmf.nmf_init(A, z(40, 5), z(30, 6))
    yield "init 1-D W0", lambda: nmf.nmf_init(A, z(40), z(30, 1))
    yield "objective W rows", lambda: nmf.nmf_objective_dense(A, z(39, 5), z(30, 5))
    yield "features Xprev", lambda: nmf.nmf_mlp_features(G, B, Xprev=z(nrhs, k + 1))
    yield "features G", lambda: nmf.nmf_mlp_features(z(k + 1, k + 1, dtype=torch.float64), B)


def test_shape_mismatches_raise_before_launch(nmf):
    for name, call in cases(nmf):
        before = nmf.nmf_kernel_launches()
        with pytest.raises((ValueError, TypeError)):
            call()
        assert nmf.nmf_kernel_launches() == before, name


def test_network_and_handle_shape_checks(nmf):
    import synth
    k, h = 4, 8
    net = nmf.nmf_mlp_create(k, h, torch.from_numpy(synth.mlp_init(k, h)).cuda())
    A = torch.rand((40, 30), device="cuda")
    hd = nmf.nmf_init(A, torch.rand((40, k), device="cuda"), torch.rand((30, k), device="cuda"))
    calls = [
        ("forward features", lambda: net.nmf_mlp_forward(z(5, 3 * k + 1))),
        ("propose features", lambda: net.nmf_mlp_propose(z(5, 3 * k - 1))),
        ("gradient labels", lambda: net.nmf_mlp_gradient(z(5, 3 * k),
                                                         z(4, 1, dtype=torch.int64))),
        ("train labels", lambda: net.nmf_mlp_train(z(5, 3 * k), z(5, 2, dtype=torch.int64))),
        ("set_factors W", lambda: hd.nmf_set_factors(W=z(41, k))),
        ("set_factors Ht", lambda: hd.nmf_set_factors(Ht=z(30, k + 1))),
    ]
    for name, call in calls:
        before = nmf.nmf_kernel_launches()
        with pytest.raises((ValueError, TypeError)):
            call()
        assert nmf.nmf_kernel_launches() == before, name
    hd.nmf_destroy()
    net.nmf_mlp_destroy()
