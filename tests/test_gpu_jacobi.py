"""Compute plus communication: Jacobi sweeps over subdomains in a ring whose halo rows move
over multi-path transfers -- as direct launches, as transfer graphs (the paper's setup,
Sec. 5.4) and as one captured graph holding both stencil kernels and halo exchanges -- all
equal to the oracle's undivided grid, bit for bit."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
import payload
from oracle import jacobi as J
from oracle import planner as P

pytestmark = pytest.mark.gpu


class Ring:
    def __init__(self, ctx, nsub, rows, cols, seed, specs):
        import torch
        self.ctx, self.nsub, self.rows, self.cols = ctx, nsub, rows, cols
        self.grid = payload.fill("f32", seed, nsub * rows * cols * 4).view(np.float32).reshape(nsub * rows, cols)
        self.bufs = [[torch.zeros((rows + 2, cols), dtype=torch.float32, device="cuda") for _ in range(nsub)]
                     for _ in range(2)]
        for i in range(nsub):
            self.bufs[0][i][1:rows + 1].copy_(torch.from_numpy(self.grid[i * rows:(i + 1) * rows]))
        self.plan = mpt.mpt_plan(ctx, cols * 4, P.D2D, specs)
        torch.cuda.synchronize()

    def exchanges(self, b):
        """(dst, src) of every halo copy of buffer set b: first interior row to the upper
        neighbour's bottom halo, last interior row to the lower neighbour's top halo."""
        out, n, r = [], self.nsub, self.rows
        for i in range(n):
            out.append((self.bufs[b][(i - 1) % n][r + 1].data_ptr(), self.bufs[b][i][1].data_ptr()))
            out.append((self.bufs[b][(i + 1) % n][0].data_ptr(), self.bufs[b][i][r].data_ptr()))
        return out

    def sweep(self, b, stream):
        for i in range(self.nsub):
            mpt.mpt_demo_jacobi_step(self.bufs[b][i], self.bufs[1 - b][i], self.rows, self.cols, stream)

    def result(self, b):
        import torch
        torch.cuda.synchronize()
        return np.concatenate([self.bufs[b][i][1:self.rows + 1].cpu().numpy() for i in range(self.nsub)])


SPECS = [(P.CE, 32768, 4096), (P.SM, 32768, 4096)]


@pytest.mark.parametrize("mode", ["eager", "graphs", "captured"])
def test_ring_jacobi_equals_undivided_grid(mode):
    import torch
    ctx = mpt.mpt_ctx_create(0)
    ring = Ring(ctx, 4, 8, 4099, 0x5EED0006, SPECS)
    s = torch.cuda.Stream()
    iters = 6
    # initial halos
    for dst, src in ring.exchanges(0):
        mpt.mpt_launch_eager(ctx, ring.plan, dst, src, s)
    handles = {}
    if mode == "graphs":
        handles = {b: [mpt.mpt_capture(ctx, ring.plan, d, sp) for d, sp in ring.exchanges(b)] for b in (0, 1)}
    if mode == "captured":
        handles = {b: [mpt.mpt_prepare(ctx, ring.plan, d, sp, mpt.MPT_PREPARE_EAGER) for d, sp in ring.exchanges(b)]
                   for b in (0, 1)}
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            for b in (0, 1):  # two sweeps: 0 -> 1 then 1 -> 0
                ring.sweep(b, s)
                for h in handles[1 - b]:
                    mpt.mpt_launch(h, s)
        for _ in range(iters // 2):
            g.replay()
    else:
        for it in range(iters):
            b = it % 2
            ring.sweep(b, s)
            if mode == "eager":
                for dst, src in ring.exchanges(1 - b):
                    mpt.mpt_launch_eager(ctx, ring.plan, dst, src, s)
            else:
                for h in handles[1 - b]:
                    mpt.mpt_launch(h, s)
    s.synchronize()
    got = ring.result(iters % 2)
    want = J.run(ring.grid, iters)
    assert np.array_equal(got, want), f"max diff {np.abs(got - want).max()}"
    for hs in handles.values():
        for h in hs:
            mpt.mpt_graph_release(h)
    mpt.mpt_plan_destroy(ring.plan)
    assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK
    mpt.mpt_ctx_destroy(ctx)


def test_staged_path_refuses_first_use_inside_capture():
    import torch
    ctx = mpt.mpt_ctx_create(0)
    a = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    plan = mpt.mpt_plan(ctx, 1 << 20, P.D2D, [(P.HS, 65536, 256 * 1024)])
    h = mpt.mpt_prepare(ctx, plan, b.data_ptr(), a.data_ptr(), mpt.MPT_PREPARE_EAGER)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(mpt.MptError):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            mpt.mpt_launch(h, s)
    # after one run outside a capture the staging exists and capturing works
    torch.cuda.synchronize()
    mpt.mpt_launch(h, torch.cuda.current_stream())
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s, capture_error_mode="thread_local"):
        mpt.mpt_launch(h, s)
    a.fill_(9)
    g2.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    mpt.mpt_graph_release(h)
    mpt.mpt_plan_destroy(plan)
    mpt.mpt_ctx_destroy(ctx)


@pytest.mark.parametrize("rows,cols,offset", [
    (1, 4, 0), (1, 8, 0), (2, 1024, 0), (8, 4096, 0), (3, 8192 + 4, 0), (33, 1028, 0), (5, 256 * 4 * 3 + 12, 0),
    (8, 4099, 0), (5, 2, 0), (7, 3, 0), (4, 4096, 1),  # scalar kernel: ragged columns, misaligned rows
])
def test_single_sweep_matches_oracle(rows, cols, offset):
    """One mpt_demo_jacobi_step on a (rows + 2) x cols subdomain against the oracle's sweep
    of the same rows (bit-exact, fp32 in the stated order); halo rows of `out` untouched.
    cols % 4 == 0 on 16-byte aligned rows takes the column-strip kernel, the rest the
    one-thread-per-point kernel."""
    import torch
    grid = payload.fill("f32", 0x5EED0007 + rows * 131 + cols, (rows + 2) * cols * 4).view(np.float32)
    grid = grid.reshape(rows + 2, cols)
    n = (rows + 2) * cols
    buf_in = torch.zeros(n + offset, dtype=torch.float32, device="cuda")
    buf_out = torch.full((n + offset + 8,), 7.0, dtype=torch.float32, device="cuda")
    buf_in[offset:offset + n].copy_(torch.from_numpy(grid.reshape(-1)))
    assert mpt.mpt_demo_jacobi_step(buf_in[offset:], buf_out[offset:], rows, cols,
                                    torch.cuda.current_stream()) is None
    torch.cuda.synchronize()
    got = buf_out[offset:offset + n].cpu().numpy().reshape(rows + 2, cols)
    want = J.step(grid)[1:rows + 1]
    assert np.array_equal(got[1:rows + 1], want), f"max diff {np.abs(got[1:rows + 1] - want).max()}"
    assert (got[0] == 7.0).all() and (got[rows + 1] == 7.0).all()
    assert (buf_out[offset + n:].cpu().numpy() == 7.0).all()
