"""Helpers shared by the GPU tests: move a generated instance to the device,
run the C-ABI path, and fetch results as numpy arrays."""
import numpy as np

import datagen


def device_inputs(inst, perm_seed, table=False):
    """(offsets, tids, perm) on the device; perm is the caller-made table of
    datagen.permutations when `table`, else None (the library computes its
    permutations from params.perm_seed)."""
    import torch
    dev = torch.device("cuda:0")
    off = torch.from_numpy(inst.offsets.astype(np.int64)).to(dev)
    tids = torch.from_numpy(inst.tids.astype(np.int32)).to(dev)
    perm = (torch.from_numpy(datagen.permutations(inst.m, perm_seed).astype(np.int32)).to(dev) if table
            else None)
    return off, tids, perm


def seeded_params(perm_seed, params=None):
    """Build parameters (defaults, or a copy of `params`) with perm_seed set."""
    import paper_1102_1003_gb300 as pkg
    p = pkg.batmap_default_params()
    if params is not None:
        for k, _ in params._fields_:
            setattr(p, k, getattr(params, k))
    p.perm_seed = int(perm_seed)
    return p


def run_all_pairs(inst, s=None, perm_seed=0, params=None, want_full=True, table=False):
    """Build + pair_support_all; returns (full uint32 packed or None, n_out, pairs uint32[k,3], set).
    The permutations are the library's for seed perm_seed, or the caller-made table."""
    import torch
    import paper_1102_1003_gb300 as pkg
    off, tids, perm = device_inputs(inst, perm_seed, table)
    bset = pkg.batmap_build(inst.m, off, tids, perm, params=seeded_params(perm_seed, params))
    npairs = inst.n * (inst.n - 1) // 2
    full = torch.empty(max(npairs, 1), dtype=torch.int32, device="cuda") if want_full else None
    n_out, pairs = pkg.pair_support_all(bset, inst.s if s is None else s, full=full)
    torch.cuda.synchronize()
    f = full[:npairs].cpu().numpy().astype(np.uint32) if want_full else None
    return f, n_out, pairs.cpu().numpy().astype(np.uint32).reshape(-1, 3), bset


def layout_errors(inst, bset, perm_seed, c_num=2, c_den=1, table=False):
    """Check every item's BatMap against the definition (hash ranges from the
    load factor c = c_num / c_den, the permutations of seed perm_seed: the
    oracle's restatement of the library's generator, or the caller-made
    table); returns a list of errors."""
    import paper_1102_1003_gb300 as pkg
    from oracle import batmap_rules as R
    from oracle import permutation as OP
    lay = pkg.batmap_export_layout(bset)
    info = lay["info"]
    perms = datagen.permutations(inst.m, perm_seed) if table else OP.permutations(inst.m, perm_seed, 3)
    s = info["shift"]
    r0 = info["r0"]
    errs = []
    if s != R.shift_bits(inst.m, 7) or r0 != 1 << s:
        errs.append(f"shift {s} / r0 {r0} differ from the sizing rule")
    fo = lay["fail_offsets"].astype(np.int64)
    for i in range(inst.n):
        r = int(lay["range"][i])
        size = len(inst.tidlist(i))
        if r != R.hash_range(size, r0, c_num, c_den):
            errs.append(f"item {i}: r={r} but the rule gives {R.hash_range(size, r0, c_num, c_den)}")
            continue
        b0 = int(lay["byte_offset"][i])
        bm = lay["bytes"][b0:b0 + 3 * r]
        f = lay["fail_tids"][fo[i]:fo[i + 1]]
        if f.size > 1 and not (np.diff(f.astype(np.int64)) > 0).all():
            errs.append(f"item {i}: F_i not sorted")
        e = R.check_layout(bm, inst.tidlist(i), f, perms, r, r0, s)
        errs.extend(f"item {i}: {x}" for x in e)
    return errs
