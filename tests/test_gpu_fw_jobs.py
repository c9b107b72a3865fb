"""General block products of the forward operator on the tensor cores (the
persistent kernel behind the sibling and interpolation blocks with
fw_engine = FDS_FW_TENSOR): rectangular blocks, both op(A) = A and A^H,
gathered rows of x and scattered rows of y, set and accumulate, blocks wider
than 128 complex columns (several passes), empty and one-column blocks, all
against complex128 products."""
import numpy as np
import pytest

from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu


def _jobs(rng, shapes, nx, ny):
    """Random blocks (m, k, op, set) with disjoint y rows and random x rows."""
    A, meta, maps = [], [], []
    aoff = 0
    yfree = rng.permutation(ny)
    ypos = 0
    for (m, k, op, st, xm, ym) in shapes:
        stored = (k, m) if op else (m, k)
        a = (rng.standard_normal(stored) + 1j * rng.standard_normal(stored)) * np.logspace(-6, 6, stored[0])[:, None]
        A.append(a)
        lda = max(1, stored[0])
        if xm:
            xmap = rng.choice(nx, k, replace=False).astype(np.int32)
            xo, xrow = len(maps), 0
            maps.extend(xmap.tolist())
        else:
            xrow = int(rng.integers(0, nx - k + 1))
            xmap, xo = np.arange(xrow, xrow + k), -1
        if ym:
            rows = yfree[ypos:ypos + m]
            ypos += m
            yo, yrow = len(maps), 0
            maps.extend(rows.tolist())
            yrows = rows
        else:
            # contiguous rows: take a fresh contiguous range past the mapped ones
            yo, yrow = -1, None
            yrows = None
        meta.append(dict(m=m, k=k, op=op, set=st, aoff=aoff, lda=lda, xrow=xrow, xo=xo, xrows=np.asarray(xmap),
                         yrow=yrow, yo=yo, yrows=yrows))
        aoff += a.size
    return A, meta, maps


@pytest.mark.parametrize("nc", [1, 33, 100])
def test_jobs_match_complex128(nc):
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(7 + nc)
    # (m, k, op, set, x mapped, y mapped)
    shapes = [(56, 56, 0, 0, 1, 1), (64, 64, 1, 1, 1, 1), (65, 129, 0, 0, 1, 1), (130, 37, 1, 1, 0, 1),
              (1, 1, 0, 0, 0, 1), (200, 300, 1, 0, 1, 1), (17, 0, 0, 1, 0, 1), (28, 36, 0, 0, 1, 0),
              (36, 28, 1, 1, 0, 0), (128, 128, 0, 0, 0, 0)]
    nx = 1200
    nmapped = sum(s[0] for s in shapes if s[5])
    ncontig = sum(s[0] for s in shapes if not s[5])
    ny = nmapped + ncontig
    A, meta, maps = _jobs(rng, [s for s in shapes], nx, nmapped)
    # contiguous y ranges after the mapped rows
    pos = nmapped
    for q in meta:
        if q["yo"] < 0:
            q["yrow"], q["yrows"] = pos, np.arange(pos, pos + q["m"])
            pos += q["m"]
    X = (rng.standard_normal((nx, nc)) + 1j * rng.standard_normal((nx, nc))) * np.logspace(-3, 3, nc)[None, :]
    Y0 = rng.standard_normal((ny, nc)) + 1j * rng.standard_normal((ny, nc))
    dA = torch.tensor(np.concatenate([a.T.ravel() for a in A]), device="cuda")
    dX = torch.tensor(np.ascontiguousarray(X.T), device="cuda")
    dY = torch.tensor(np.ascontiguousarray(Y0.T), device="cuda")
    g = lambda key: [q[key] for q in meta]
    fds.fds_zgemm_jobs_tc(g("m"), g("k"), g("op"), g("aoff"), g("lda"), g("xrow"), g("xo"), g("yrow"), g("yo"),
                          g("set"), np.array(maps, np.int32), dA, dX, dY)
    got = dY.cpu().numpy().T
    touched = np.zeros(ny, bool)
    for a, q in zip(A, meta):
        opA = a.conj().T if q["op"] else a
        xs = X[q["xrows"]] if q["k"] else np.zeros((0, nc))
        prod = opA @ xs if q["k"] else np.zeros((q["m"], nc), complex)
        base = 0 if q["set"] else Y0[q["yrows"]]
        scale = np.abs(opA) @ np.abs(xs) if q["k"] else np.zeros((q["m"], nc))
        bound = 2e-11 * scale + 4e-14 * np.abs(base + prod) + 1e-300
        excess = np.abs(got[q["yrows"]] - base - prod) / bound
        assert excess.max() <= 1.0, (q["m"], q["k"], q["op"], q["set"], excess.max())
        touched[q["yrows"]] = True
    # rows no job addresses are untouched
    assert np.array_equal(got[~touched], Y0[~touched])


def test_jobs_equal_leaf_kernel_on_leaf_blocks():
    # square contiguous blocks: the general kernel and the leaf kernel cut the
    # same slices and add the same exact accumulators
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(5)
    d = np.array([128, 1, 64, 127, 100, 128], np.int32)
    nc = 70
    As = [(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))) * np.logspace(-8, 8, k)[:, None] for k in d]
    D = int(d.sum())
    off = np.concatenate([[0], np.cumsum(d)])
    X = rng.standard_normal((D, nc)) + 1j * rng.standard_normal((D, nc))
    Y0 = rng.standard_normal((D, nc)) + 1j * rng.standard_normal((D, nc))
    dA = torch.tensor(np.concatenate([a.T.ravel() for a in As]), device="cuda")
    dX = torch.tensor(np.ascontiguousarray(X.T), device="cuda")
    dY1 = torch.tensor(np.ascontiguousarray(Y0.T), device="cuda")
    dY2 = dY1.clone()
    fds.fds_zgemm_blocks_tc(d, dA, dX, dY1)
    aoff = np.concatenate([[0], np.cumsum(d.astype(np.int64) ** 2)])[:-1]
    n = len(d)
    fds.fds_zgemm_jobs_tc(d, d, np.zeros(n), aoff, d, off[:-1], -np.ones(n), off[:-1], -np.ones(n), np.zeros(n),
                          None, dA, dX, dY2)
    y1, y2 = dY1.cpu().numpy(), dY2.cpu().numpy()
    assert np.abs(y1 - y2).max() <= 1e-15 * np.abs(y1).max()
