"""GB300-native stencil engine (arxiv 2603.00477): C-ABI library + thin binding.

``paper_2603_00477_gb300.binding`` wraps ``libgbstencil.so`` (built from
``csrc/`` by ``paper_2603_00477_gb300.build``); ``inputs`` holds the seeded
synthetic input generators.  Importing the package loads nothing compiled.
"""

__all__ = ["binding", "build", "inputs"]
