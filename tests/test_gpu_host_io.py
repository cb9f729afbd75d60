"""pp_grad_host: the evaluation of pp_grad on host buffers.  Pinned buffers are read
and written in place by the kernels, pageable ones staged through the workspace;
either way the kernels and their arithmetic are those of pp_grad, so the results
must equal pp_grad's bit for bit (E up to the order of its FP64 atomic sum).  Also
checked against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import series as O  # noqa: E402
from paper_2307_12041_gb300 import binding, synth  # noqa: E402

from test_gpu_parity import nerr  # noqa: E402


def _host(a, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.pin_memory() if pinned else t.clone()


def _outs(n, pinned):
    mk = (lambda k, dt: torch.empty(k, dtype=dt).pin_memory()) if pinned else (lambda k, dt: torch.empty(k, dtype=dt))
    return mk(n, torch.float32), mk(n, torch.float32), mk(n, torch.float32), mk(1, torch.float64)


CASES = [(0, None), (1, 20_000)]      # 2,000 blocks x 64^2; 20,000 blocks x 512^2 (SM-pair kernel)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
@pytest.mark.parametrize("pinned_in,pinned_out", [(True, True), (False, False), (True, False), (False, True)])
def test_host_buffers_give_pp_grad_bit_for_bit(case, prec, pinned_in, pinned_out):
    p = synth.workload(*case)
    dev = torch.device("cuda")
    x, y, w, h, c = binding.to_device(p, dev)
    ref = binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    hin = [_host(a, pinned_in) for a in (p.x, p.y, p.w, p.h)]
    hc = None if p.c is None else _host(p.c, pinned_in)
    out = _outs(p.n, pinned_out)
    got = binding.grad_host(*hin, hc, p.W, p.H, p.Mx, p.My, prec, out=out)
    torch.cuda.synchronize()
    binding.sync_status()
    for k in range(3):
        assert torch.equal(got[k], ref[k].cpu()), (prec, k)
    # E is an FP64 sum of CTA partials added atomically: equal up to their order
    assert abs(got[3].item() - ref[3].item()) <= 1e-13 * abs(ref[3].item())


def test_host_buffers_match_the_oracle():
    p = synth.workload(0)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    hin = [_host(a, True) for a in (p.x, p.y, p.w, p.h)]
    hc = None if p.c is None else _host(p.c, True)
    gx, gy, N, E = binding.grad_host(*hin, hc, p.W, p.H, p.Mx, p.My, "fp32")
    torch.cuda.synchronize()
    assert nerr(gx.numpy().astype(np.float64), ref["gx"]) < 2e-6
    assert nerr(gy.numpy().astype(np.float64), ref["gy"]) < 2e-6
    assert nerr(N.numpy().astype(np.float64), ref["N"]) < 2e-6
    assert abs(E.item() - ref["E"]) <= 2e-6 * abs(ref["E"])


def test_device_inputs_host_outputs_and_empty_placement():
    p = synth.workload(0)
    dev = torch.device("cuda")
    x, y, w, h, c = binding.to_device(p, dev)
    ref = binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "tf32")
    # device tensors are accepted where host ones are expected (binding passes pointers)
    import ctypes
    prob = binding.make_problem(x, y, w, h, c, p.W, p.H, p.Mx, p.My)
    out = _outs(p.n, True)
    need = binding.lib().pp_grad_host_workspace_size(ctypes.byref(prob), binding.PRECISIONS["tf32"])
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    st = binding.lib().pp_grad_host(ctypes.byref(prob), binding.PRECISIONS["tf32"], binding.SAMPLES["rect"],
                                    out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), out[3].data_ptr(),
                                    ws.data_ptr(), ws.numel(), binding._stream_handle(dev))
    assert st == 0, binding.lib().pp_last_error()
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(out[k], ref[k].cpu())
    # n = 0: E = 0, nothing else touched
    e = torch.full((1,), 7.0, dtype=torch.float64).pin_memory()
    z = torch.empty(0, dtype=torch.float32)
    binding.grad_host(z, z, z, z, None, p.W, p.H, p.Mx, p.My, "tf32",
                      out=(z, z, None, e))
    torch.cuda.synchronize()
    assert e.item() == 0.0


def test_host_call_rejects_bad_arguments():
    import ctypes
    p = synth.workload(0)
    hin = [_host(a, True) for a in (p.x, p.y, p.w, p.h)]
    out = _outs(p.n, True)
    prob = binding.Problem(p.W, p.H, p.n, hin[0].data_ptr(), hin[1].data_ptr(), hin[2].data_ptr(),
                           hin[3].data_ptr(), None, p.Mx, p.My)
    L = binding.lib()
    dev = torch.device("cuda")
    need = L.pp_grad_host_workspace_size(ctypes.byref(prob), 1)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    h = binding._stream_handle(dev)
    # workspace one byte short
    assert L.pp_grad_host(ctypes.byref(prob), 1, 0, out[0].data_ptr(), out[1].data_ptr(), None, None,
                          ws.data_ptr(), need - 1, h) != 0
    # gx missing
    assert L.pp_grad_host(ctypes.byref(prob), 1, 0, None, out[1].data_ptr(), None, None,
                          ws.data_ptr(), need, h) != 0
    # misaligned input
    bad = binding.Problem(p.W, p.H, p.n - 1, hin[0].data_ptr() + 2, hin[1].data_ptr(), hin[2].data_ptr(),
                          hin[3].data_ptr(), None, p.Mx, p.My)
    assert L.pp_grad_host(ctypes.byref(bad), 1, 0, out[0].data_ptr(), out[1].data_ptr(), None, None,
                          ws.data_ptr(), need, h) != 0
    assert "aligned" in L.pp_last_error().decode()
