"""Child process of test_gpu_debug_bounds.py: loads the bounds-check build
(FEM_DEBUG_BOUNDS=1 must be set before the package is imported) and prints one
JSON line with what it saw.  Not a test module by itself."""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import meshgen  # noqa: E402
import oracle  # noqa: E402
from helpers import TOL_FP64, TOL_MIXED, oracle_K, rel_err, rounded_inputs  # noqa: E402


def main():
    from paper_1501_04784_gb300 import _build, abi
    assert _build.DEBUG_BOUNDS, "FEM_DEBUG_BOUNDS=1 must be set"
    _build.build()
    from paper_1501_04784_gb300 import fem
    out = {"lib": abi.library_path(), "clean": {}, "planted": None, "after": None}

    def dev(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)

    meshes = {"hex": (8, meshgen.hex_grid(7, 5, 3, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True)),
              "tet": (4, meshgen.kuhn_tets(6, 4, 3, jitter=0.3, seed=2, permute_nodes=True, permute_elems=True))}
    # every path of the patch kernels under the checks: fused builds in both
    # precisions, the staged (integrate, then assemble) path, the batched kernel;
    # none may report a bad index
    for name, (npe, m) in meshes.items():
        for prec, tol in (("fp64", TOL_FP64), ("mixed", TOL_MIXED)):
            X, c = rounded_inputs(m, prec)
            dt = torch.float64 if prec == "fp64" else torch.float32
            Xd, cd = dev(X, dt), dev(c, dt)
            ref = oracle_K(m, X, c)
            mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=64)
            fused = mesh.build_K(Xd, cd, prec).cpu().numpy()
            mesh.sync()
            ke = mesh.integrate_local(Xd, cd, prec)
            staged = mesh.assemble_csr(ke, prec).cpu().numpy()
            mesh.sync()
            twin = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=64)
            batched = fem.build_K_batched([mesh, twin], [Xd, Xd], [cd, cd], prec)
            mesh.sync()
            out["clean"][f"{name}_{prec}"] = bool(
                rel_err(fused, ref["vals"], ref["cs"]) <= tol and rel_err(staged, ref["vals"], ref["cs"]) <= tol
                and all(np.array_equal(b.cpu().numpy(), fused) for b in batched))
    # the elasticity operator's patch kernel, fused and staged
    for name, (npe, m) in meshes.items():
        lame = meshgen.lame(m)
        X32, c32 = m.X.astype(np.float32), lame.astype(np.float32)
        ref = oracle.build_K(npe, X32.astype(np.float64), m.E, c32.astype(np.float64), op="elasticity")
        mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=48,
                        operator_kind=2)
        Xd, cd = dev(X32, torch.float32), dev(c32, torch.float32)
        fused = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
        mesh.sync()
        staged = mesh.assemble_csr(mesh.integrate_local(Xd, cd, "mixed"), "mixed").cpu().numpy()
        mesh.sync()
        out["clean"][f"{name}_elastic"] = bool(rel_err(fused, ref["vals"], ref["cs"]) <= TOL_MIXED
                                               and rel_err(staged, ref["vals"], ref["cs"]) <= TOL_MIXED)
    # one planted out-of-range node id per block: caught, skipped, reported once
    npe, m = meshes["hex"]
    X, c = rounded_inputs(m, "mixed")
    Xd, cd = dev(X, torch.float32), dev(c, torch.float32)
    planted = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), debug_stall=2)
    planted.build_K(Xd, cd, "mixed")
    try:
        planted.sync()
        out["planted"] = "FEM_OK"
    except abi.FemError as e:
        out["planted"] = e.name
    planted.sync()  # the status word was cleared
    # the context stays usable
    ok = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    vals = ok.build_K(Xd, cd, "mixed").cpu().numpy()
    ok.sync()
    ref = oracle_K(m, X, c)
    out["after"] = bool(rel_err(vals, ref["vals"], ref["cs"]) <= TOL_MIXED)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
