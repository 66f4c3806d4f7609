"""The tiled variant-B MD step (spread mode "tiles") against the row gather,
the all-atomic spreading and the oracle.

Every path hands the same fixed-point transfers to the nodes (Sec. 3, Eqs.
(7), (8)) and evaluates the coupling force (Eqs. (4)-(6)) with the same
arithmetic, so whole runs must agree bit for bit; the oracle then bounds all
of them at the parity tolerances.  The cases cover ragged tiles (lattice rows
not a multiple of the 4 x 4 tile), the periodic wrap of the halo rows, the
shortest lattices the path accepts (6 rows), rows of 512 nodes (16 active
words), tiles whose records do not fit in shared memory, many particles
leaving their rows within a cycle, particles added between cycles, graph
replay and a save / restore in the middle.
"""
import numpy as np
import pytest

from gpu_common import TOL, assert_pops_close, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu


def _periodic_diff(a, b, shape):
    d = a - b
    L = np.array(shape, dtype=float)
    return d - L * np.round(d / L)


def _run(shape, n, spread, precision="fp32", n_sub=5, cycles=2, kT=1e-4, zeta=1.5, seed=41, vel_scale=1.0,
         region=None, graph=False):
    g = lbmd.LBMD(*shape, variant="B", precision=precision, n_sub=n_sub, kT=kT, zeta=zeta, seed=seed,
                  max_particles=n, spread=spread)
    pos = inputs.uniform_positions(n, shape if region is None else region, seed)
    vel = vel_scale * inputs.maxwell_velocities(n, kT, seed)
    g.add_particles(pos, vel)
    if graph:
        g.run_cycles(cycles)
    else:
        g.cycle(cycles)
    out = (g.populations(), *g.particles(), g.node_field())
    g.close()
    return out, pos, vel


def _assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(24, 20, 18), (40, 6, 6), (33, 13, 7)])
def test_tiles_rows_atomic_bitwise_and_oracle(precision, shape):
    n = 12 * shape[1] * shape[2]
    runs = {}
    for spread in ("tiles", "rows", "atomic"):
        runs[spread], pos, vel = _run(shape, n, spread, precision)
    _assert_same(runs["tiles"], runs["rows"])
    _assert_same(runs["tiles"], runs["atomic"])
    o, _ = pair(shape, precision=precision, variant="B", n_sub=5, kT=1e-4, zeta=1.5, seed=41)
    o.add_particles(pos, vel)
    o.cycle(2)
    assert_pops_close(runs["tiles"][0], o.populations(), precision)
    po, vo = o.particles()
    assert np.abs(_periodic_diff(runs["tiles"][1], po, shape)).max() <= TOL[precision] * max(shape)
    assert_vec_close(runs["tiles"][2], vo, precision, "velocities")
    o.close()


def test_rows_of_512_nodes():
    shape, n = (512, 7, 9), 12 * 63
    _assert_same(_run(shape, n, "tiles")[0], _run(shape, n, "rows")[0])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tiles_beyond_shared_memory(precision):
    # dense particles: a tile's 36 staged rows hold more active nodes than
    # its shared memory (every tile, then only some: a dense slab)
    shape = (512, 8, 8)
    n = 4000
    _assert_same(_run(shape, n, "tiles", precision)[0], _run(shape, n, "rows", precision)[0])
    region = (512, 8, 1)  # particles only in z < 1: some tiles staged, some not
    _assert_same(_run(shape, n, "tiles", precision, region=region)[0],
                 _run(shape, n, "rows", precision, region=region)[0])


def test_many_particles_leave_their_rows():
    # fast particles: a large share crosses a row (or moves within its row to
    # a cell whose corners are not active) within every cycle
    shape, n = (32, 24, 20), 6000
    a = _run(shape, n, "tiles", kT=1e-3, zeta=0.2, n_sub=10, cycles=3, vel_scale=8.0)[0]
    b = _run(shape, n, "rows", kT=1e-3, zeta=0.2, n_sub=10, cycles=3, vel_scale=8.0)[0]
    _assert_same(a, b)


@pytest.mark.parametrize("n_sub", [5, 10])
def test_graph_replay_and_added_particles(n_sub):
    # replayed cycles equal eager ones for odd and even n_sub (the position and
    # record buffers flip every MD step), also after particles are added
    shape, n = (24, 20, 18), 8000
    runs = {}
    for mode in ("eager", "graph", "rows"):
        g = lbmd.LBMD(*shape, variant="B", n_sub=n_sub, kT=1e-4, zeta=1.5, seed=7, max_particles=n,
                      spread="rows" if mode == "rows" else "tiles")
        for k in range(2):
            m = n // 2
            g.add_particles(inputs.uniform_positions(m, shape, 7 + k), inputs.maxwell_velocities(m, 1e-4, 7 + k))
            if mode == "graph":
                g.run_cycles(2)
            else:
                g.cycle(2)
        runs[mode] = (g.populations(), *g.particles(), g.node_field())
        g.close()
    _assert_same(runs["graph"], runs["eager"])
    _assert_same(runs["eager"], runs["rows"])


def test_save_and_restore_mid_run():
    shape, n = (24, 20, 18), 5000
    pos, vel = inputs.uniform_positions(n, shape, 9), inputs.maxwell_velocities(n, 1e-4, 9)

    def make():
        return lbmd.LBMD(*shape, variant="B", n_sub=5, kT=1e-4, zeta=1.5, seed=9, max_particles=n, spread="tiles")

    g = make()
    g.add_particles(pos, vel)
    g.run_cycles(2)
    state = g.save_state()
    g.run_cycles(2)
    want = (g.populations(), *g.particles())
    g.close()
    h = make()
    h.load_state(state)
    h.run_cycles(2)
    _assert_same((h.populations(), *h.particles()), want)
    h.close()


def test_tiles_at_the_benchmark_density():
    # 15 particles per row, as in the benchmark: the same bits as the row
    # gather that AUTO picks there
    shape = (64, 32, 32)
    n = 15 * 32 * 32
    _assert_same(_run(shape, n, "tiles")[0], _run(shape, n, "auto")[0])
