"""Checkpoint / resume: running G generations equals running G/2, saving the
whole state to a host blob, loading it into a fresh handle and running G/2
more -- for a plain dual-island run, a surrogate-screened run (ring buffer,
network weights, Adam moments and step count included) and a batch of
uneven instances.  Integer results, so equality is exact; the network's
parameters are compared bit for bit (every kernel of the training step is
deterministic).  Blobs of another shape or instance are refused before
anything is written."""
import numpy as np
import pytest
import torch

from ffs_workloads import make_batch, make_instance

pytestmark = pytest.mark.gpu


def _islands_state(gpu, isl):
    out = []
    for i in range(isl.n_islands):
        pop, ms = gpu.island_tensors(isl, i)
        torch.cuda.synchronize()
        out.append((pop.cpu().numpy(), ms.cpu().numpy()))
    return out


def _assert_same_islands(gpu, a, b):
    sa, sb = _islands_state(gpu, a), _islands_state(gpu, b)
    for i, ((pa, ma), (pb, mb)) in enumerate(zip(sa, sb)):
        assert np.array_equal(pa, pb), i
        assert np.array_equal(ma, mb), i
    assert a.generation() == b.generation()
    assert gpu.ffs_islands_decoded(a) == gpu.ffs_islands_decoded(b)
    assert gpu.ffs_islands_best(a) == gpu.ffs_islands_best(b)


def _dual(gpu, inst, mode=1, gap=3):
    prm = gpu.ffs_params_default()
    prm.migration_mode, prm.migration_gap = mode, gap
    return gpu.Islands(inst, prm, 2, 8, 8, 2, 64)


@pytest.mark.parametrize("mode", [1, 2])
def test_islands_checkpoint_resume_equals_uninterrupted_run(gpu, mode):
    spec = make_instance(30, 6, 2, 4, seed=31)
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    G = 10
    a = _dual(gpu, inst, mode)
    gpu.ffs_island_step(a, -1, G // 2)
    blob = gpu.ffs_checkpoint_save(a)
    gpu.ffs_island_step(a, -1, G - G // 2)
    b = _dual(gpu, inst, mode)
    gpu.ffs_island_step(b, -1, 2)          # some other state, overwritten by the load
    gpu.ffs_checkpoint_load(b, blob)
    assert b.generation() == G // 2
    gpu.ffs_island_step(b, -1, G - G // 2)
    _assert_same_islands(gpu, a, b)


@pytest.mark.parametrize("overlap,screen_pseudo", [(0, 0), (1, 0), (1, 1)])
def test_screened_islands_checkpoint_resume_equals_uninterrupted_run(gpu, overlap, screen_pseudo):
    spec = make_instance(40, 6, 2, 5, seed=41)
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    rows = cols = 8
    K = 4

    def make(net_seed):
        prm = gpu.ffs_params_default()
        prm.migration_mode, prm.migration_gap = 1, 4
        isl = gpu.Islands(inst, prm, 1, rows, cols, 1, 64)
        net = gpu.MLP(540, 512, 256, 1024)
        net.init(net_seed)
        sp = gpu.ffs_surrogate_params_default()
        sp.candidates, sp.warmup_generations, sp.train_every, sp.train_steps = K, 2, 1, 2
        sp.train_batch, sp.ring_capacity = 128, 512      # the ring wraps within the run
        sp.overlap = overlap
        sp.screen_pseudo = screen_pseudo
        gpu.ffs_islands_attach_surrogate(isl, net, sp)
        return isl, net

    a, net_a = make(3)
    gpu.ffs_island_step(a, -1, 6)
    blob = gpu.ffs_checkpoint_save(a)
    gpu.ffs_island_step(a, -1, 6)
    b, net_b = make(99)                    # other weights: the load must bring the saved ones
    gpu.ffs_checkpoint_load(b, blob)
    gpu.ffs_island_step(b, -1, 6)
    _assert_same_islands(gpu, a, b)
    assert net_a.adam_steps() == net_b.adam_steps() > 0
    for which in (0, 2, 3):
        pa, pb = net_a.get(which=which), net_b.get(which=which)
        for k in pa:
            assert np.array_equal(np.asarray(pa[k]), np.asarray(pb[k])), (which, k)
    sa = np.zeros(rows * cols * K, np.float32)
    sb = np.zeros(rows * cols * K, np.float32)
    pairs_a = gpu.ffs_islands_surrogate_last(a, sa)
    pairs_b = gpu.ffs_islands_surrogate_last(b, sb)
    torch.cuda.synchronize()
    assert pairs_a == pairs_b and np.array_equal(sa, sb)
    # a plain handle cannot take a screened checkpoint
    plain = gpu.Islands(inst, gpu.ffs_params_default(), 1, rows, cols, 1, 64)
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_checkpoint_load(plain, blob)
    assert e.value.status == gpu.FFS_EINVAL


def test_islands_checkpoint_refuses_other_shapes_and_instances(gpu):
    spec = make_instance(30, 6, 2, 4, seed=31)
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    a = _dual(gpu, inst)
    gpu.ffs_island_step(a, -1, 2)
    blob = gpu.ffs_checkpoint_save(a)
    other = make_instance(30, 6, 2, 4, seed=32)
    oinst = gpu.Instance(other.n, other.S, other.M, other.p)
    before = _islands_state(gpu, _dual(gpu, oinst))
    b = _dual(gpu, oinst)
    for bad in (blob, blob[:100], blob[:len(blob) // 2]):
        with pytest.raises(gpu.FFSError) as e:
            gpu.ffs_checkpoint_load(b, bad)
        assert e.value.status == gpu.FFS_EINVAL
    after = _islands_state(gpu, b)
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(before, after))
    c = gpu.Islands(inst, gpu.ffs_params_default(), 1, 8, 8, 1, 64)
    with pytest.raises(gpu.FFSError):
        gpu.ffs_checkpoint_load(c, blob)


def test_checkpoints_refuse_corrupted_blobs(gpu):
    """A checkpoint with one byte altered (in the header, a population row, a
    makespan or the surrogate's ring and weights) fails its checksum: load
    returns FFS_EINVAL and writes nothing; the unaltered blob still loads."""
    spec = make_instance(30, 6, 2, 4, seed=31)
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    a = _dual(gpu, inst)
    net = gpu.MLP(540, 512, 256, 1024)
    net.init(3)
    sp = gpu.ffs_surrogate_params_default()
    sp.candidates, sp.train_batch, sp.ring_capacity, sp.warmup_generations = 4, 128, 1024, 1
    gpu.ffs_islands_attach_surrogate(a, net, sp)
    gpu.ffs_island_step(a, -1, 3)
    blob = gpu.ffs_checkpoint_save(a)
    b = _dual(gpu, inst)
    net_b = gpu.MLP(540, 512, 256, 1024)
    gpu.ffs_islands_attach_surrogate(b, net_b, sp)
    before = _islands_state(gpu, b)
    for at in (40, 300, len(blob) // 3, len(blob) // 2, len(blob) - 5):
        bad = blob.copy()
        bad[at] ^= 0x10
        with pytest.raises(gpu.FFSError) as e:
            gpu.ffs_checkpoint_load(b, bad)
        assert e.value.status == gpu.FFS_EINVAL
    after = _islands_state(gpu, b)
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(before, after))
    gpu.ffs_checkpoint_load(b, blob)
    _assert_same_islands(gpu, a, b)
    # the batch's checkpoint likewise
    specs = make_batch(count=3, seed=5, n_range=(5, 40), s_range=(2, 5), m_range=(1, 4))
    bt = gpu.Batch(specs, gpu.ffs_params_default(), 8, 8)
    gpu.ffs_batch_step(bt, 2)
    bblob = gpu.ffs_batch_checkpoint_save(bt)
    bad = bblob.copy()
    bad[len(bad) // 2] ^= 0x01
    bt2 = gpu.Batch(specs, gpu.ffs_params_default(), 8, 8)
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_batch_checkpoint_load(bt2, bad)
    assert e.value.status == gpu.FFS_EINVAL
    gpu.ffs_batch_checkpoint_load(bt2, bblob)


def _reseal(blob, bytes_at, sum_at, length=None):
    """The blob with its length field (at byte `bytes_at`) set to `length` when
    given and its checksum (at `sum_at`) recomputed over that length: FNV-1a
    over the 64-bit words, the checksum's own word taken as zero -- so that
    only the checks after the checksum can refuse it."""
    b = blob.copy()
    if length is not None:
        b[bytes_at:bytes_at + 8] = np.frombuffer(np.int64(length).tobytes(), np.uint8)
    n = int(np.frombuffer(b[bytes_at:bytes_at + 8].tobytes(), np.int64)[0])
    words = np.frombuffer(b[:n].tobytes(), dtype=np.uint64).copy()
    words[sum_at // 8] = 0
    h = 14695981039346656037
    for w in words.tolist():
        h = ((h ^ w) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    b[sum_at:sum_at + 8] = np.frombuffer(np.uint64(h).tobytes(), np.uint8)
    return b


def test_checkpoints_read_only_their_own_length_and_check_parameters(gpu):
    """Bytes after a blob's own length are never read (a longer buffer loads);
    a length field made shorter, with a valid checksum over that length, is
    refused because the sections no longer fit; GA parameters outside
    ffs_islands_create's limits are refused under a valid checksum; nothing
    is written by a refused load."""
    spec = make_instance(24, 5, 2, 3, seed=32)
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    a = _dual(gpu, inst)
    gpu.ffs_island_step(a, -1, 4)
    blob = gpu.ffs_checkpoint_save(a)
    BYTES, SUM, PRM = 40, 48, 56   # IslandsBlobHeader offsets
    assert np.array_equal(_reseal(blob, BYTES, SUM), blob)   # the test's checksum is the library's
    b = _dual(gpu, inst)
    before = _islands_state(gpu, b)
    refused = [_reseal(blob, BYTES, SUM, len(blob) - 16)]
    for field, value in (("migration_mode", 9), ("ring_den", 0), ("theta_num", 1 << 40), ("migration_gap", -1)):
        bad = blob.copy()
        f = getattr(gpu.ffs_params, field)
        bad[PRM + f.offset:PRM + f.offset + f.size] = np.frombuffer(
            np.array([value], dtype=np.int64 if f.size == 8 else np.int32).tobytes(), np.uint8)
        refused.append(_reseal(bad, BYTES, SUM))
    for bad in refused:
        with pytest.raises(gpu.FFSError) as e:
            gpu.ffs_checkpoint_load(b, bad)
        assert e.value.status == gpu.FFS_EINVAL
    after = _islands_state(gpu, b)
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(before, after))
    gpu.ffs_checkpoint_load(b, np.concatenate([blob, np.full(64, 0xA5, np.uint8)]))
    _assert_same_islands(gpu, a, b)
    # the batch's blob likewise (BatchBlobHeader: length at 48, checksum at 56)
    specs = make_batch(count=3, seed=6, n_range=(5, 40), s_range=(2, 5), m_range=(1, 4))
    bt = gpu.Batch(specs, gpu.ffs_params_default(), 8, 8)
    gpu.ffs_batch_step(bt, 2)
    bblob = gpu.ffs_batch_checkpoint_save(bt)
    assert np.array_equal(_reseal(bblob, 48, 56), bblob)
    bt2 = gpu.Batch(specs, gpu.ffs_params_default(), 8, 8)
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_batch_checkpoint_load(bt2, _reseal(bblob, 48, 56, len(bblob) - 16))
    assert e.value.status == gpu.FFS_EINVAL
    gpu.ffs_batch_checkpoint_load(bt2, np.concatenate([bblob, np.zeros(32, np.uint8)]))
    assert gpu.ffs_batch_best(bt2).tolist() == gpu.ffs_batch_best(bt).tolist()


def test_screened_checkpoint_checks_the_network_before_writing(gpu):
    """The network's part of a screened blob (its last section) is checked
    before anything is written: with its magic altered and the checksum
    resealed, the load is refused and the islands keep their rows."""
    spec = make_instance(20, 4, 2, 3, seed=33)
    inst = gpu.Instance(spec.n, spec.S, spec.M, spec.p)
    sp = gpu.ffs_surrogate_params_default()
    sp.candidates, sp.train_batch, sp.ring_capacity, sp.warmup_generations = 4, 128, 1024, 1
    a = _dual(gpu, inst)
    net = gpu.MLP(540, 512, 256, 1024)
    net.init(5)
    gpu.ffs_islands_attach_surrogate(a, net, sp)
    gpu.ffs_island_step(a, -1, 3)
    blob = gpu.ffs_checkpoint_save(a)
    net_bytes = int(gpu.load().ffs_mlp_state_bytes(net.handle))
    at = len(blob) - (net_bytes + 15) // 16 * 16   # the network's header
    bad = blob.copy()
    bad[at] ^= 0x01
    bad = _reseal(bad, 40, 48)
    b = _dual(gpu, inst)
    net_b = gpu.MLP(540, 512, 256, 1024)
    gpu.ffs_islands_attach_surrogate(b, net_b, sp)
    before = _islands_state(gpu, b)
    with pytest.raises(gpu.FFSError) as e:
        gpu.ffs_checkpoint_load(b, bad)
    assert e.value.status == gpu.FFS_EINVAL and "network state" in str(e.value)
    after = _islands_state(gpu, b)
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(before, after))
    gpu.ffs_checkpoint_load(b, blob)
    _assert_same_islands(gpu, a, b)


_ALLOC_CHILD = """
import sys
sys.path.insert(0, {root!r})
import paper_1903_10722_gb300 as gpu
try:
    gpu.MLP(540, 512, 256, 256)
    print("no failure")
except gpu.FFSError as e:
    print("status", e.status)
m = gpu.MLP(540, 512, 256, 256)   # later allocations succeed
m.init(1)
print("after", m.adam_steps())
"""


def test_allocation_failure_is_reported(gpu):
    """An allocation made to fail on the host (FFS_INJECT_ALLOC_FAILURE=3: the
    third allocation of a network's buffers, in a child process) is reported
    as FFS_ENOMEM with everything allocated so far freed; the next network is
    created and used normally."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FFS_INJECT_ALLOC_FAILURE="3")
    r = subprocess.run([sys.executable, "-c", _ALLOC_CHILD.format(root=root)], capture_output=True, text=True,
                       env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "status %d" % gpu.FFS_ENOMEM in r.stdout and "after 0" in r.stdout, r.stdout


def test_batch_checkpoint_resume_equals_uninterrupted_run(gpu):
    specs = make_batch(count=7, seed=5, n_range=(5, 120), s_range=(2, 9), m_range=(1, 8))
    prm = gpu.ffs_params_default()
    a = gpu.Batch(specs, prm, 6, 6)
    gpu.ffs_batch_step(a, 4)
    blob = gpu.ffs_batch_checkpoint_save(a)
    gpu.ffs_batch_step(a, 5)
    b = gpu.Batch(specs, prm, 6, 6)
    gpu.ffs_batch_checkpoint_load(b, blob)
    assert b.info()["generation"] == 4
    gpu.ffs_batch_step(b, 5)
    for i in range(len(specs)):
        pa, ma = gpu.batch_tensors(a, i)
        pb, mb = gpu.batch_tensors(b, i)
        torch.cuda.synchronize()
        assert torch.equal(pa, pb) and torch.equal(ma, mb), i
    assert gpu.ffs_batch_decoded(a) == gpu.ffs_batch_decoded(b)
    assert np.array_equal(gpu.ffs_batch_best(a), gpu.ffs_batch_best(b))
    # another torus or other instances: refused
    c = gpu.Batch(specs, prm, 6, 5)
    with pytest.raises(gpu.FFSError):
        gpu.ffs_batch_checkpoint_load(c, blob)
    d = gpu.Batch(make_batch(count=7, seed=6, n_range=(5, 120), s_range=(2, 9), m_range=(1, 8)), prm, 6, 6)
    with pytest.raises(gpu.FFSError):
        gpu.ffs_batch_checkpoint_load(d, blob)


def test_batch_set_then_step_matches_get(gpu):
    """ffs_batch_set writes rows and makespans that ffs_batch_get reads back."""
    specs = make_batch(count=3, seed=8, n_range=(5, 40), s_range=(2, 5), m_range=(1, 4))
    b = gpu.Batch(specs, gpu.ffs_params_default(), 4, 4)
    pop, ms = gpu.batch_tensors(b, 1)
    flipped = torch.flip(pop, dims=[0]).contiguous()
    ms2 = torch.flip(ms, dims=[0]).contiguous()
    gpu.ffs_batch_set(b, 1, flipped, specs[1].n, ms2)
    back, bms = gpu.batch_tensors(b, 1)
    torch.cuda.synchronize()
    assert torch.equal(back, flipped) and torch.equal(bms, ms2)
