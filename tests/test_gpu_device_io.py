"""The device-pointer boundary calls (swe_state_init_device,
swe_state_set_device, swe_copy_out_device, swe_grad_device,
swe_tape_gauges_device) through the C ABI with torch CUDA buffers: each
gives bitwise the results of its host-array counterpart, and each is
ordered after the work the caller queued on its own stream."""
import numpy as np
import pytest

from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built
from test_oracle_tangent import smooth_wet_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = torch.device("cuda", 0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def ptrs(*ts):
    return [None if t is None else t.data_ptr() for t in ts]


def host_fields(st):
    return st.fields()


def device_fields(st, T, stream=None):
    out = [torch.full((T,), np.nan, dtype=torch.float64, device=DEV) for _ in range(3)]
    t, m = st.copy_out_device(*ptrs(*out), stream=stream)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out], t, m


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kernel", ["tiled", "edge"])
def test_init_set_and_copy_out_on_device_equal_the_host_calls(prec, kernel):
    ensure_built()
    c = inputs.random_flow_case(nx=37, ny=23, seed=41)
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision=prec, kernel=kernel)
    a = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    d = [dev(x) for x in (c.h, c.hu, c.hv, c.z, c.n)]
    b = swe.State.from_device(mesh, *ptrs(*d))
    assert a.next_dt() == b.next_dt()
    a.run(25)
    b.run(25)
    ha = host_fields(a)
    hb, t, m = device_fields(b, mesh.T)
    for x, y in zip(ha, hb):
        assert np.array_equal(x, y)
    assert (t, m) == a.copy_out()
    # set from device buffers, then step again
    a.set(c.h, c.hu, c.hv)
    b.set_device(*ptrs(*d[:3]))
    a.run(7)
    b.run(7)
    for x, y in zip(host_fields(a), device_fields(b, mesh.T)[0]):
        assert np.array_equal(x, y)
    # a constant Manning n from the device call
    e = swe.State.from_device(mesh, *ptrs(*d[:4]), None, manning_const=0.03)
    f = swe.State(mesh, c.h, c.hu, c.hv, c.z, None, manning_const=0.03)
    e.run(5)
    f.run(5)
    for x, y in zip(host_fields(f), device_fields(e, mesh.T)[0]):
        assert np.array_equal(x, y)


def test_copy_out_device_of_an_ensemble_whose_scenarios_end_in_different_buffers():
    ensure_built()
    cases = [inputs.random_flow_case(nx=12 + 3 * i, ny=8 + i, seed=50 + i) for i in range(4)]
    mesh = swe.Mesh.ensemble([(c.mesh.xy, c.mesh.tri) for c in cases], precision="f64")
    cat = lambda k: np.concatenate([getattr(c, k) for c in cases])
    st = swe.State(mesh, cat("h"), cat("hu"), cat("hv"), cat("z"), cat("n"))
    st.advance(1.5)
    steps = {st.scenario(i)["steps"] % 2 for i in range(len(cases))}
    assert steps == {0, 1}
    got, t, m = device_fields(st, mesh.T)
    for x, y in zip(host_fields(st), got):
        assert np.array_equal(x, y)


def test_device_calls_wait_for_the_callers_stream():
    """Inputs written on a side stream and passed with that stream are read
    only after the writes (no host synchronisation in between)."""
    ensure_built()
    c = inputs.random_flow_case(nx=300, ny=200, lx=3_000.0, ly=2_000.0, seed=61)  # 120,000 cells
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision="f64")
    ref = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    src = [dev(x) for x in (c.h, c.hu, c.hv, c.z, c.n)]
    torch.cuda.synchronize()
    side = torch.cuda.Stream(device=DEV)
    dst = [torch.zeros_like(x) for x in src]
    with torch.cuda.stream(side):
        torch.cuda._sleep(20_000_000)  # keep the side stream busy before the copies
        for x, y in zip(dst, src):
            x.copy_(y)
    st = swe.State.from_device(mesh, *ptrs(*dst), stream=side.cuda_stream)
    ref.run(5)
    st.run(5)
    for x, y in zip(host_fields(ref), host_fields(st)):
        assert np.array_equal(x, y)


def test_gradient_with_device_seeds_and_outputs_equals_the_host_call():
    ensure_built()
    c = smooth_wet_case(seed=2)
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision="f64")
    st = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    gauges = [3, 40, 77]
    N = 11
    tape = swe.Tape(st, N, 4, gauges)
    rng = np.random.default_rng(3)
    T = mesh.T
    g = [rng.standard_normal(T) for _ in range(3)] + [rng.standard_normal((N, len(gauges)))]
    want = tape.grad(*g)
    seeds = [dev(x) for x in g]
    outs = [torch.empty(T, dtype=torch.float64, device=DEV) for _ in range(5)]
    tape.grad_device(ptrs(*seeds), ptrs(*outs))
    for k, o in zip(("h", "hu", "hv", "z", "n"), outs):
        assert np.array_equal(o.cpu().numpy(), want[k]), k
    gh = torch.empty((N, len(gauges)), dtype=torch.float64, device=DEV)
    tape.gauges_device(gh.data_ptr())
    assert np.array_equal(gh.cpu().numpy(), tape.gauge_h)
    # seeds may be left out, as in the host call
    tape.grad_device([None, None, None, seeds[3].data_ptr()], ptrs(*outs))
    want2 = tape.grad(g_gauge=g[3])
    assert np.array_equal(outs[4].cpu().numpy(), want2["n"])


def test_autograd_on_cuda_tensors_equals_the_cpu_tensor_path():
    ensure_built()
    from paper_1807_00672_gb300 import grad as sgrad
    c = smooth_wet_case(seed=5)
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision="f64")
    res = {}
    for where in ("cpu", "cuda"):
        x = [torch.tensor(a, device=where, requires_grad=True) for a in (c.h, c.hu, c.hv, c.z, c.n)]
        h, hu, hv, gh = sgrad.rollout(mesh, *x, n_steps=8, checkpoint_every=3, gauges=[4, 60])
        loss = (gh ** 2).sum() + 0.3 * (h * hv).sum()
        loss.backward()
        res[where] = [h.detach().cpu().numpy(), gh.detach().cpu().numpy()] + \
            [t.grad.cpu().numpy() for t in x]
    for a, b in zip(res["cpu"], res["cuda"]):
        assert np.array_equal(a, b)
