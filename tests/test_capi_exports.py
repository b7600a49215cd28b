"""The C-ABI library loads without a GPU and exports every symbol of include/map_smoother.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_13319_gb300 import _binding, build
    build.build()
    return _binding.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "map_smoother.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(map_(?:smoother|batch|fma)_\w+)\s*\(", text)))


def test_header_and_binding_agree():
    from paper_2512_13319_gb300 import _binding
    assert declared_functions() == sorted(_binding.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    from paper_2512_13319_gb300 import _binding as B
    assert B.map_smoother_version()
    assert B.map_smoother_supported(B.MAP_MODEL_LINEAR, 4, 2, B.MAP_FP32)
    assert B.map_smoother_supported(B.MAP_MODEL_COORD_TURN, 5, 2, B.MAP_FP64)
    assert not B.map_smoother_supported(B.MAP_MODEL_LINEAR, 7, 7, B.MAP_FP32)
    assert not B.map_smoother_supported(B.MAP_MODEL_LINEAR, 4, 2, 9)


def test_create_rejects_bad_descriptors_before_touching_the_device(lib):
    from paper_2512_13319_gb300 import _binding as B
    from paper_2512_13319_gb300 import synth
    model = synth.wiener_velocity(2)
    cases = [
        (dict(T=0), B.MAP_ERR_SHAPE),
        (dict(dt=-1.0), B.MAP_ERR_INVALID_ARG),
        (dict(precision=7), B.MAP_ERR_INVALID_ARG),
    ]
    for kw, status in cases:
        args = dict(T=10, dt=0.01)
        args.update(kw)
        T, dt = args.pop("T"), args.pop("dt")
        d, keep = B.make_desc(model, T, dt, **args)
        with pytest.raises(B.MapError) as ei:
            B.map_smoother_create(d)
        assert ei.value.status == status
    d, keep = B.make_desc(model, 10, 0.01)
    d.nx = 9
    with pytest.raises(B.MapError) as ei:
        B.map_smoother_create(d)
    assert ei.value.status == B.MAP_ERR_SHAPE
