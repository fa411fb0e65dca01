"""GB300-native laminographic filtered backprojection.

Importing the package loads nothing; ``paper_2401_11101_gb300.lamino`` is the
binding of the CUDA library and ``paper_2401_11101_gb300.inputs`` the seeded
synthetic input generators.
"""
