"""B300-native GATE traffic-engineering iteration engine.

The compute path lives in the C-ABI library ``libte.so`` (CUDA, sm_103a);
``paper_2605_01748_b300.te`` is its thin Python binding and
``paper_2605_01748_b300.instances`` generates seeded synthetic inputs.
Submodules are imported explicitly so that the instance generator can be used
on hosts without a GPU.
"""
__all__ = ["te", "instances", "build"]
